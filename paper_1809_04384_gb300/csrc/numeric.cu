// Numeric stages of the hybrid DH^2 construction and the DH^2 matvec.
//
//   analytic stage (Section 2): Chebyshev nodes in the padded boxes, leaf bases
//     v_{tc,i nu} = int phi_i exp(i kappa <x,c>) L_{t,nu}(x) (3-point rule),
//     transfer matrices E_{t'c} (Eq. nested_apx) as three m x m factors, the
//     nearfield blocks (Eq. 2), couplings S_b = g_c(xi_t, xi_s) generated where
//     they are used (never stored);
//   Section 3.2: basis weights R (bottom-up QR), block weights 1/|G_b|_F, total
//     weights Z-hat (top-down QR of the stacked blocks, rows and columns),
//     truncation (bottom-up SVD: Gram matrix + Hermitian Jacobi in FP64),
//     projection S~_b = C_tc S_b C_sc^* (Lemma "Projections");
//   matvec: forward transform (column basis), couplings, backward transform
//     (row basis), nearfield (derived from Eq. nested and Eq. vsw).
//
// T is the working precision: float for DH2_MIXED, double for DH2_FP64.
#include <algorithm>
#include <cmath>
#include <map>
#include <exception>
#include <mutex>
#include <thread>
#include <array>
#include <string>

#include "numeric.cuh"
#include "tcgen05.cuh"

namespace dh2 {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kThreads = 256;

// Device error word: kernels that meet a non-finite value set a bit instead of trapping;
// the host reads the word after each stage and returns DH2_ENUMERIC.
enum : unsigned {
    ERR_TSQR_NONFINITE = 1u, ERR_TRUNC_NONFINITE = 2u, ERR_TSQR_INPUT = 4u, ERR_STACK_NONFINITE = 8u,
    ERR_KRON_NONFINITE = 16u, ERR_TC_TIMEOUT = 32u,
    ERR_RANK_CAP = 64u   // not an error: a truncation rank exceeded its learned cap (the pass is redone)
};
__device__ __forceinline__ void raise_err(unsigned* err, unsigned bit) { atomicOr(err, bit); }

// ----------------------------------------------------------------------------- math wrappers

__device__ __forceinline__ void sc(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sc(double x, double* s, double* c) { sincos(x, s, c); }

// exp(i kappa r) / (4 pi r) for a difference vector d
template <class T>
__device__ __forceinline__ cx<T> helmholtz_d(T dx, T dy, T dz, T kappa) {
    T r2 = dx * dx + dy * dy + dz * dz;
    T r = sqrt(r2);
    T s, c;
    sc(kappa * r, &s, &c);
    T f = T(1) / (T(4.0 * kPi) * r);
    return cx<T>{c * f, s * f};
}

// Lagrange polynomial l_j of the m nodes xi at x (product form)
__device__ __forceinline__ double lagrange1(const double* xi, int m, int j, double x) {
    double v = 1.0;
    for (int i = 0; i < m; ++i)
        if (i != j) v *= (x - xi[i]) / (xi[j] - xi[i]);
    return v;
}

// derivative of the Lagrange polynomial l_j of the m nodes xi at x (product rule):
// l_j'(x) = sum_{q != j} 1 / (xi_j - xi_q) prod_{i != j, q} (x - xi_i) / (xi_j - xi_i)
__device__ __forceinline__ double lagrange1_d(const double* xi, int m, int j, double x) {
    double s = 0.0;
    for (int q = 0; q < m; ++q) {
        if (q == j) continue;
        double v = 1.0 / (xi[j] - xi[q]);
        for (int i = 0; i < m; ++i)
            if (i != j && i != q) v *= (x - xi[i]) / (xi[j] - xi[i]);
        s += v;
    }
    return s;
}

// d/dn_y g(x, y) = exp(i kappa r) (1 - i kappa r) <x - y, n_y> / (4 pi r^3) for d = x - y
template <class T>
__device__ __forceinline__ cx<T> dlp_d(T dx, T dy, T dz, T n0, T n1, T n2, T kappa) {
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T r = sqrt(r2);
    T s, c;
    sc(kappa * r, &s, &c);
    const T kr = kappa * r;
    const T f = (dx * n0 + dy * n1 + dz * n2) / (T(4.0 * kPi) * r2 * r);
    return cx<T>{(c + kr * s) * f, (s - kr * c) * f};
}

// ----------------------------------------------------------------------------- analytic stage

// nodes[t][a][j] = mid_a + half_a cos(pi (2j+1) / (2m)), half padded to >= 1e-3 max half
__global__ void k_cheb_nodes(const double* __restrict__ lo, const double* __restrict__ hi, int32_t nc,
                             int m, double* nodes) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc) return;
    double mid[3], half[3], hmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        mid[a] = (lo[a * nc + t] + hi[a * nc + t]) * 0.5;
        half[a] = (hi[a * nc + t] - lo[a * nc + t]) * 0.5;
        hmax = fmax(hmax, half[a]);
    }
    for (int a = 0; a < 3; ++a) {
        double h = fmax(half[a], 1e-3 * hmax);
        for (int j = 0; j < m; ++j)
            nodes[((int64_t)t * 3 + a) * m + j] = mid[a] + h * cos(kPi * (2 * j + 1) / (2.0 * m));
    }
}

struct LeafTask {
    int32_t t, gdir, off, rows;
    int64_t voff;
};

// unit normals of the elements (original order): n = (v1 - v0) x (v2 - v0) / |.| (vertex order)
__global__ void k_normals(const double* __restrict__ vert, const int32_t* __restrict__ tri, int64_t n,
                          double* __restrict__ nrm) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double* a = vert + 3 * (int64_t)tri[3 * e];
    const double* b = vert + 3 * (int64_t)tri[3 * e + 1];
    const double* c = vert + 3 * (int64_t)tri[3 * e + 2];
    const double u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
    const double v0 = c[0] - a[0], v1 = c[1] - a[1], v2 = c[2] - a[2];
    const double x = u1 * v2 - u2 * v1, y = u2 * v0 - u0 * v2, z = u0 * v1 - u1 * v0;
    const double inv = 1.0 / sqrt(x * x + y * y + z * z);
    nrm[3 * e] = x * inv;
    nrm[3 * e + 1] = y * inv;
    nrm[3 * e + 2] = z * inv;
}

// Leaf bases (FP64, stored as T).  Row basis V_tc (W = false):
//   v_{i nu} = |T_i|/3 sum_q exp(i kappa <x_q, c>) L_{t,nu}(x_q);
// column basis of the double layer W_tc (W = true), the normal derivative of the same
// functions along the element normal n_i:
//   w_{i nu} = |T_i|/3 sum_q exp(i kappa <x_q, c>) (i kappa <n_i, c> L_{t,nu}(x_q) + <n_i, grad L_{t,nu}(x_q)>).
template <class T, bool W>
__global__ void k_leaf_basis(const LeafTask* __restrict__ tasks, const int32_t* __restrict__ perm,
                             const double* __restrict__ area, const double* __restrict__ x3,
                             const double* __restrict__ nodes, const double* __restrict__ dirs,
                             int m, double kappa, const double* __restrict__ nrm, cx<T>* V) {
    const LeafTask tk = tasks[blockIdx.x];
    const int k = m * m * m;
    __shared__ double xi[3][8];
    if (threadIdx.x < 3 * m) xi[threadIdx.x / m][threadIdx.x % m] = nodes[((int64_t)tk.t * 3) * m + threadIdx.x];
    __syncthreads();
    const double c0 = dirs[3 * tk.gdir], c1 = dirs[3 * tk.gdir + 1], c2 = dirs[3 * tk.gdir + 2];
    for (int idx = threadIdx.x; idx < tk.rows * k; idx += blockDim.x) {
        int i = idx / k, nu = idx % k;
        int nx = nu % m, ny = (nu / m) % m, nz = nu / (m * m);
        int e = perm[tk.off + i];
        double w = area[e] / 3.0;
        double ar = 0.0, ai = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double* x = x3 + ((int64_t)e * 3 + q) * 3;
            const double lx = lagrange1(xi[0], m, nx, x[0]), ly = lagrange1(xi[1], m, ny, x[1]),
                         lz = lagrange1(xi[2], m, nz, x[2]);
            const double L = lx * ly * lz;
            double s, c;
            sincos(kappa * (x[0] * c0 + x[1] * c1 + x[2] * c2), &s, &c);
            if constexpr (W) {
                const double n0 = nrm[3 * e], n1 = nrm[3 * e + 1], n2 = nrm[3 * e + 2];
                const double dn = n0 * lagrange1_d(xi[0], m, nx, x[0]) * ly * lz +
                                  n1 * lx * lagrange1_d(xi[1], m, ny, x[1]) * lz +
                                  n2 * lx * ly * lagrange1_d(xi[2], m, nz, x[2]);
                const double kl = kappa * (n0 * c0 + n1 * c1 + n2 * c2) * L;   // imaginary part of the factor
                ar += c * dn - s * kl;
                ai += s * dn + c * kl;
            } else {
                ar += c * L;
                ai += s * L;
            }
        }
        V[tk.voff + idx] = cx<T>{T(w * ar), T(w * ai)};
    }
}

struct TransferTask {
    int32_t t, ts, gdir, gdir_son;
    int64_t eoff;
};

// factors of E_{t'c}: E_a[nu'][nu] = exp(i kappa xi_{t',a,nu'} (c_a - c'_a)) l_{t,a,nu}(xi_{t',a,nu'})
template <class T>
__global__ void k_transfer(const TransferTask* __restrict__ tasks, const double* __restrict__ nodes,
                           const double* __restrict__ dirs, int m, double kappa, cx<T>* E) {
    const TransferTask tk = tasks[blockIdx.x];
    const int mm = m * m;
    for (int idx = threadIdx.x; idx < 3 * mm; idx += blockDim.x) {
        int a = idx / mm, r = idx % mm;
        int nup = r / m, nu = r % m;
        const double* xt = nodes + ((int64_t)tk.t * 3 + a) * m;
        double xs = nodes[((int64_t)tk.ts * 3 + a) * m + nup];
        double dc = dirs[3 * tk.gdir + a] - dirs[3 * tk.gdir_son + a];
        double L = lagrange1(xt, m, nu, xs);
        double s, c;
        sincos(kappa * xs * dc, &s, &c);
        E[tk.eoff + idx] = cx<T>{T(c * L), T(s * L)};
    }
}

// ----------------------------------------------------------------------------- nearfield

struct NearSeg {
    int32_t rows, cols, roff, coff;   // cluster-order ranges
    int32_t ld;                       // panel width of the row leaf
    int32_t pad;
    int64_t poff;                     // panel offset of (row 0, first column of this segment)
    int64_t cpos;                     // where the segment's column indices go in the panel's list
};

// split of an FP64 coordinate into float hi + lo (for differences in FP32)
__global__ void k_split_quad(const int32_t* __restrict__ perm, const double* __restrict__ x3, int64_t n,
                             float* qh, float* ql) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * 9) return;
    int64_t r = idx / 9, w = idx % 9;
    double v = x3[(int64_t)perm[r] * 9 + w];
    float h = (float)v;
    qh[idx] = h;
    ql[idx] = (float)(v - (double)h);
}

__global__ void k_cluster_quad(const int32_t* __restrict__ perm, const double* __restrict__ x3, int64_t n,
                               double* out) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * 9) return;
    int64_t r = idx / 9, w = idx % 9;
    out[idx] = x3[(int64_t)perm[r] * 9 + w];
}

template <class T>
struct QuadRows;   // quadrature nodes in cluster order

template <>
struct QuadRows<float> {
    const float* h;
    const float* l;
    __device__ __forceinline__ void diff(int64_t r, int p, int64_t c, int q, float* d) const {
        for (int a = 0; a < 3; ++a) {
            int64_t i = r * 9 + p * 3 + a, j = c * 9 + q * 3 + a;
            d[a] = (h[i] - h[j]) + (l[i] - l[j]);
        }
    }
};
template <>
struct QuadRows<double> {
    const double* x;      // [n][3][3] cluster order
    __device__ __forceinline__ void diff(int64_t r, int p, int64_t c, int q, double* d) const {
        for (int a = 0; a < 3; ++a) d[a] = x[r * 9 + p * 3 + a] - x[c * 9 + q * 3 + a];
    }
};

__constant__ double c_w7[7];

// Nearfield entries by quadrature: single layer (DLP = false) g_ij as in Eq. (2), the
// diagonal by the 7-point rule in x against the 3-point rule in y; double layer (DLP = true)
// the normal derivative along the column element's normal, 3 x 3 rule, 0 on the diagonal.
template <class T, bool DLP>
__global__ void k_nearfield(const NearSeg* __restrict__ segs, QuadRows<T> qr,
                            const int32_t* __restrict__ perm, const double* __restrict__ area,
                            const double* __restrict__ x3, const double* __restrict__ x7, double kappa,
                            const double* __restrict__ nrm, cx<T>* P, int32_t* colidx) {
    const NearSeg sg = segs[blockIdx.x];
    const T kap = (T)kappa;
    // the panel's column -> x~ index list, read by the matvec
    for (int j = threadIdx.x; j < sg.cols; j += blockDim.x) colidx[sg.cpos + j] = sg.coff + j;
    for (int idx = threadIdx.x; idx < sg.rows * sg.cols; idx += blockDim.x) {
        int i = idx / sg.cols, j = idx % sg.cols;
        int64_t r = sg.roff + i, c = sg.coff + j;
        int e = perm[r], f = perm[c];
        cx<T> v;
        if (DLP && e == f) {
            v = zero<T>();
        } else if (e != f) {
            T acc_r = 0, acc_i = 0;
            T n0 = 0, n1 = 0, n2 = 0;
            if constexpr (DLP) {
                n0 = T(nrm[3 * f]);
                n1 = T(nrm[3 * f + 1]);
                n2 = T(nrm[3 * f + 2]);
            }
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    T d[3];
                    qr.diff(r, p, c, q, d);
                    cx<T> g;
                    if constexpr (DLP) g = dlp_d<T>(d[0], d[1], d[2], n0, n1, n2, kap);
                    else g = helmholtz_d<T>(d[0], d[1], d[2], kap);
                    acc_r += g.x;
                    acc_i += g.y;
                }
            T w = T(area[e] / 3.0 * (area[f] / 3.0));
            v = cx<T>{w * acc_r, w * acc_i};
        } else {
            // 7-point rule in x against the 3-point rule in y, FP64
            double ar = 0, ai = 0;
            for (int p = 0; p < 7; ++p)
                for (int q = 0; q < 3; ++q) {
                    const double* xp = x7 + ((int64_t)e * 7 + p) * 3;
                    const double* yq = x3 + ((int64_t)e * 3 + q) * 3;
                    cx<double> g = helmholtz_d<double>(xp[0] - yq[0], xp[1] - yq[1], xp[2] - yq[2], kappa);
                    double w = c_w7[p] / 3.0;
                    ar += w * g.x;
                    ai += w * g.y;
                }
            double a2 = area[e] * area[e];
            v = cx<T>{T(a2 * ar), T(a2 * ai)};
        }
        P[sg.poff + (int64_t)i * sg.ld + j] = v;
    }
}

// ----------------------------------------------------------------------------- coupling generator

// S_b[nu][mu] = g_c(xi_{t,nu}, xi_{s,mu}) from per-axis tables in shared memory:
// D[a][i][j] = xi_{t,a,i} - xi_{s,a,j} and P[a][i][j] = D[a][i][j] c_a (evaluated in FP64),
// and index tables dn[nu], dm[mu] that hold the three per-axis table offsets of a node in
// 10-bit fields, so that dn[nu] + dm[mu] packs the offsets of the pair (no division by m).
template <class T>
struct SGen {
    const T* D;
    const T* P;
    const uint32_t* dn;
    const uint32_t* dm;
    T kappa;
    __device__ __forceinline__ cx<T> operator()(int nu, int mu) const {
        const uint32_t u = dn[nu] + dm[mu];
        const int ix = u & 1023u, iy = (u >> 10) & 1023u, iz = u >> 20;
        return value(D[ix], D[iy], D[iz], P[ix] + P[iy] + P[iz]);
    }
    // exp(i kappa (r - p)) / (4 pi r), r = |d|
    __device__ __forceinline__ cx<T> value(T dx, T dy, T dz, T p) const;
};

// FP32: r from the reciprocal square root; the phase is brought to [-pi, pi] by Cody and
// Waite's two-constant reduction (2 pi split into a float head and the float of the
// remainder), after which the hardware sine and cosine are accurate to about 4e-7.
template <>
__device__ __forceinline__ cx<float> SGen<float>::value(float dx, float dy, float dz, float p) const {
    constexpr double k2pi = 2.0 * kPi;
    constexpr float hi = (float)k2pi;
    constexpr float lo = (float)(k2pi - (double)hi);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ri = rsqrtf(r2);
    const float ph = kappa * (r2 * ri - p);
    const float j = rintf(ph * (float)(1.0 / k2pi));
    float red = fmaf(-j, hi, ph);
    red = fmaf(-j, lo, red);
    float s, c;
    __sincosf(red, &s, &c);
    const float f = ri * (float)(1.0 / (4.0 * kPi));
    return cx<float>{c * f, s * f};
}

template <>
__device__ __forceinline__ cx<double> SGen<double>::value(double dx, double dy, double dz, double p) const {
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    double s, c;
    sincos(kappa * (r - p), &s, &c);
    const double f = 1.0 / (4.0 * kPi * r);
    return cx<double>{c * f, s * f};
}

// shared memory of the generator tables: D, P (3 m^2 each), dn, dm (m^3 each)
template <class T>
__host__ __device__ inline size_t sgen_smem_bytes(int m) {
    return 2 * 3 * (size_t)m * m * sizeof(T) + 2 * (size_t)m * m * m * sizeof(uint32_t);
}

template <class T>
__device__ SGen<T> load_sgen_tables(int32_t t, int32_t s, const double* __restrict__ cdir,
                                    const double* __restrict__ nodes, int m, double kappa, unsigned char* sm) {
    const int mm = m * m, k = mm * m;
    T* D = reinterpret_cast<T*>(sm);
    T* P = D + 3 * mm;
    uint32_t* dn = reinterpret_cast<uint32_t*>(P + 3 * mm);
    uint32_t* dm = dn + k;
    for (int idx = threadIdx.x; idx < 3 * mm; idx += blockDim.x) {
        int a = idx / mm, r = idx % mm, i = r / m, j = r % m;
        double d = nodes[((int64_t)t * 3 + a) * m + i] - nodes[((int64_t)s * 3 + a) * m + j];
        D[idx] = (T)d;
        P[idx] = (T)(d * cdir[a]);
    }
    for (int nu = threadIdx.x; nu < k; nu += blockDim.x) {
        const uint32_t nx = nu % m, ny = (nu / m) % m, nz = nu / mm;
        dn[nu] = nx * m | (mm + ny * m) << 10 | (2 * mm + nz * m) << 20;
        dm[nu] = nx | ny << 10 | nz << 20;
    }
    __syncthreads();
    return SGen<T>{D, P, dn, dm, (T)kappa};
}

// ----------------------------------------------------------------------------- stacked rows

struct BlockRowTask {
    int32_t b;         // admissible block id
    int32_t other;     // active pair whose weight R multiplies S (rows pass: s, cols pass: t)
    int32_t own;       // active pair of the other side (rows pass: t; for |G_b|)
    int32_t own_leaf;  // rows pass: the row cluster is a leaf (rows projected onto its basis);
                       // cols pass, 2: the column cluster is a leaf and K_b is not stored:
                       // rows w K_b recomputed here (other = the s pair, own = the t pair)
    int64_t dst;       // element offset of the first row in the stack
    int64_t koff;      // rows pass: where K_b = R_t S_b R_s^* is stored
};

// ----------------------------------------------------------------------------- tensor-core products

// Products on the tcgen05 tensor cores in 3xTF32 (k <= 128, FP32 data).  A complex product
// D = X Y (M = 128 rows, N = NT columns holding the real parts in [0, RP) and the imaginary
// parts in [RP, NT), RP = NT/2) is formed as two real products into one TMEM tile,
// D = A1 B1 + A2 B2, with A1 / A2 the real / imaginary part of X and B1, B2 arranged from
// Y so that the sums land on the real and imaginary columns (see the generators below).
// Every operand is split into TF32 hi + lo and each real product is hi*hi + hi*lo + lo*hi.
// K runs in chunks of KC: the operands of a chunk are generated into shared memory
// (K-major core-matrix layout, see tcgen05.cuh) once the tensor cores are done with the
// previous chunk; one thread issues the chunk's MMAs and commits them to an mbarrier.  (Two
// buffers, with or without block-wide barriers per chunk, measured slower: the chunk has to
// shrink to 16 to fit them, and the generation of the couplings, not the MMAs, bounds it.)
template <int NT>
struct TcTile {
    static constexpr int KC = NT <= 128 ? 32 : 16;
    static constexpr int RP = NT / 2;
    // B operands use the padded layout (kmaj_off_pad): (NT/8)*32 + 4 floats per K group
    static constexpr int BSZ = (KC / 4) * ((NT / 8) * 32 + 4);
    static constexpr size_t kOperandBytes = ((size_t)4 * 128 * KC + (size_t)4 * BSZ) * sizeof(float);
};

constexpr int kTcWaitPolls = 1 << 22;

struct TcState {
    float* buf;          // operand buffer (TcTile<NT>::kOperandBytes)
    uint64_t* mbar;      // completion barrier of the chunks
    uint32_t tmem;       // TMEM base (2 NT columns)
    uint32_t phase;      // chunks committed so far
    bool ok;             // no wait has timed out
};

template <int NT>
__device__ __forceinline__ void tc_operands(float* buf, float*& A1h, float*& A1l, float*& A2h, float*& A2l,
                                            float*& B1h, float*& B1l, float*& B2h, float*& B2l) {
    constexpr int KC = TcTile<NT>::KC, BSZ = TcTile<NT>::BSZ;
    A1h = buf;
    A1l = A1h + 128 * KC;
    A2h = A1l + 128 * KC;
    A2l = A2h + 128 * KC;
    B1h = A2l + 128 * KC;
    B1l = B1h + BSZ;
    B2h = B1l + BSZ;
    B2l = B2h + BSZ;
}

// D (TMEM columns [col0, col0 + NT)) = sum over K chunks of the generated operands.
// gen.load(mu0, regs) fetches what a chunk needs from global memory into registers (the
// next chunk's fetch is in flight while this chunk's operands are formed); gen(mu0, regs,
// X1h, X1l, X2h, X2l) fills the chunk.  Both are called by every thread of the block.  All
// threads of the block must call this.
template <int NT, class GA, class GB>
__device__ void tc_product(TcState& st, uint32_t col0, int K, const GA& genA, const GB& genB) {
    constexpr int KC = TcTile<NT>::KC;
    float *A1h, *A1l, *A2h, *A2l, *B1h, *B1l, *B2h, *B2l;
    tc_operands<NT>(st.buf, A1h, A1l, A2h, A2l, B1h, B1l, B2h, B2l);
    const int nchunks = (K + KC - 1) / KC;
    typename GA::Regs ra;
    typename GB::Regs rb;
    if (nchunks > 0) {
        genA.load(0, ra);
        genB.load(0, rb);
    }
    for (int ch = 0; ch < nchunks && st.ok; ++ch) {
        typename GA::Regs na;
        typename GB::Regs nb;
        if (ch + 1 < nchunks) {
            genA.load((ch + 1) * KC, na);
            genB.load((ch + 1) * KC, nb);
        }
        if (st.phase > 0) {   // the tensor cores are done with the previous operands
            st.ok = __syncthreads_and(tc::mbar_wait(st.mbar, (st.phase - 1) & 1, kTcWaitPolls));
            if (!st.ok) break;
        }
        genA(ch * KC, ra, A1h, A1l, A2h, A2l);
        genB(ch * KC, rb, B1h, B1l, B2h, B2l);
        ra = na;
        rb = nb;
        tc::fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            constexpr uint32_t lboA = (128 / 8) * 128, lboB = (NT / 8) * 128 + 16, sbo = 128;
            const uint32_t idesc = tc::idesc_tf32(128, NT);
            const float* As[6] = {A1h, A1h, A1l, A2h, A2h, A2l};
            const float* Bs[6] = {B1h, B1l, B1h, B2h, B2l, B2h};
#pragma unroll 1
            for (int s8 = 0; s8 < KC / 8; ++s8)
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const uint64_t da = tc::sdesc(tc::smem_u32(As[q]) + s8 * 2 * lboA, lboA, sbo);
                    const uint64_t db = tc::sdesc(tc::smem_u32(Bs[q]) + s8 * 2 * lboB, lboB, sbo);
                    tc::mma_tf32(st.tmem + col0, da, db, idesc, ch > 0 || s8 > 0 || q > 0);
                }
            tc::commit(st.mbar);
        }
        ++st.phase;
    }
    // the product is complete before anyone reads it
    if (st.ok && st.phase > 0) st.ok = __syncthreads_and(tc::mbar_wait(st.mbar, (st.phase - 1) & 1, kTcWaitPolls));
    tc::fence_after_sync();
}

// ncols: TMEM columns of the CTA (a power of two, 32 ... 512), 2 NT by default
template <int NT>
__device__ void tc_begin(TcState& st, float* buf, uint64_t* mbar, uint32_t* tmem_slot, uint32_t ncols = 2 * NT) {
    if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(tmem_slot, ncols);
    if (threadIdx.x == 0) tc::mbar_init(mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    st = TcState{buf, mbar, *tmem_slot, 0u, true};
}

// releases the TMEM; after a timeout, first lets committed products finish (bounded)
template <int NT>
__device__ void tc_end(TcState& st, unsigned* err, uint32_t ncols = 2 * NT) {
    if (!st.ok) {
        if (threadIdx.x == 0) raise_err(err, ERR_TC_TIMEOUT);
        if (st.phase > 0) tc::mbar_wait(st.mbar, (st.phase - 1) & 1, kTcWaitPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(st.tmem, ncols);
}

// Operand generators.  A chunk of an M = 128 operand is written at float offset idx
// (core matrices in order); the two halves of an N = NT operand at kmaj_off_pad(i, kk, NT)
// and kmaj_off_pad(i + RP, kk, NT) (padded layout, leading byte offset (NT/8) * 128 + 16).

// Coupling operand A[nu][mu] = S(nu, mu) (rows pass) or S(mu, nu) (cols pass) from two
// node tables in shared memory: P[nu] holds the node on the row side of A, Q[mu] the node on
// the column side, both as (x, y, z, w) FP32 differences from one reference node (taken in
// FP64, so that x_P - x_Q keeps full relative accuracy), and w = +-<node - ref, c> such that
// <xi_t - xi_s, c> = P.w - Q.w.  Each thread keeps one row nu and writes four consecutive
// mu with one 16-byte store per operand array.

// Two FP32 lanes per instruction (Blackwell packed arithmetic, round to nearest per lane).
namespace f2 {
__device__ __forceinline__ uint64_t pk(float a, float b) {
    return (uint64_t)__float_as_uint(a) | ((uint64_t)__float_as_uint(b) << 32);
}
__device__ __forceinline__ float lo(uint64_t x) { return __uint_as_float((uint32_t)x); }
__device__ __forceinline__ float hi(uint64_t x) { return __uint_as_float((uint32_t)(x >> 32)); }
__device__ __forceinline__ uint64_t add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
}  // namespace f2

// The coupling values S(p, q0), S(p, q1) of one row node p, two lanes at a time:
// exp(i kappa (r - <xi_p - xi_q, c>)) / (4 pi r), r = |x_p - x_q| by rsqrt, the phase reduced
// by the two-constant Cody-Waite reduction with 2 pi (rint as (x + 1.5 * 2^23) - 1.5 * 2^23,
// exact for |x| < 2^22) before the hardware sine and cosine.
__device__ __forceinline__ void coupling_pair(float4 p, float4 q0, float4 q1, float kappa, cx<float>& v0,
                                              cx<float>& v1) {
    constexpr double k2pi = 2.0 * kPi;
    constexpr float hi = (float)k2pi;
    constexpr float lo = (float)(k2pi - (double)hi);
    constexpr float kRound = 12582912.0f;
    const uint64_t dx = f2::sub(f2::pk(p.x, p.x), f2::pk(q0.x, q1.x));
    const uint64_t dy = f2::sub(f2::pk(p.y, p.y), f2::pk(q0.y, q1.y));
    const uint64_t dz = f2::sub(f2::pk(p.z, p.z), f2::pk(q0.z, q1.z));
    const uint64_t r2 = f2::fma(dx, dx, f2::fma(dy, dy, f2::mul(dz, dz)));
    const uint64_t ri = f2::pk(rsqrtf(f2::lo(r2)), rsqrtf(f2::hi(r2)));
    const uint64_t w = f2::sub(f2::pk(p.w, p.w), f2::pk(q0.w, q1.w));
    const uint64_t ph = f2::mul(f2::pk(kappa, kappa), f2::sub(f2::mul(r2, ri), w));
    const uint64_t R2 = f2::pk(kRound, kRound);
    const uint64_t j = f2::sub(f2::add(f2::mul(ph, f2::pk((float)(1.0 / k2pi), (float)(1.0 / k2pi))), R2), R2);
    uint64_t red = f2::fma(j, f2::pk(-hi, -hi), ph);
    red = f2::fma(j, f2::pk(-lo, -lo), red);
    float s0, c0, s1, c1;
    __sincosf(f2::lo(red), &s0, &c0);
    __sincosf(f2::hi(red), &s1, &c1);
    const float c4 = (float)(1.0 / (4.0 * kPi));
    const uint64_t f = f2::mul(ri, f2::pk(c4, c4));
    const uint64_t re = f2::mul(f2::pk(c0, c1), f), im = f2::mul(f2::pk(s0, s1), f);
    v0 = cx<float>{f2::lo(re), f2::lo(im)};
    v1 = cx<float>{f2::hi(re), f2::hi(im)};
}

template <int NT>
struct GenS {
    const float4* P;   // 128 entries (row side: rows nu of this M tile)
    const float4* Q;   // k entries (column side)
    int k;             // contraction length (columns mu)
    float kappa;
    int nk;            // rows of this M tile that exist (rows nu >= nk are zero)
    struct Regs {};
    __device__ void load(int, Regs&) const {}
    __device__ void operator()(int mu0, const Regs&, float* A1h, float* A1l, float* A2h, float* A2l) const {
        constexpr int KC = TcTile<NT>::KC;
        constexpr int GROUPS = KC / 4;                          // 4-wide groups of a chunk
        constexpr int IT = 128 * GROUPS / kThreads;             // the block has kThreads threads
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int w = threadIdx.x + it * kThreads;
            const int nu = w & 127, g = w >> 7;
            const float4 p = P[nu];
            float4 h1, l1, h2, l2;
            float* ph1 = &h1.x; float* pl1 = &l1.x; float* ph2 = &h2.x; float* pl2 = &l2.x;
#pragma unroll
            for (int e = 0; e < 4; e += 2) {   // two columns per packed evaluation
                const int mu = mu0 + 4 * g + e;   // Q holds 256 entries: mu + 1 < 256 is in range
                cx<float> v0, v1;
                coupling_pair(p, Q[mu], Q[mu + 1], kappa, v0, v1);
                if (!(nu < nk && mu < k)) v0 = zero<float>();
                if (!(nu < nk && mu + 1 < k)) v1 = zero<float>();
                tc::split_tf32(v0.x, ph1[e], pl1[e]);
                tc::split_tf32(v0.y, ph2[e], pl2[e]);
                tc::split_tf32(v1.x, ph1[e + 1], pl1[e + 1]);
                tc::split_tf32(v1.y, ph2[e + 1], pl2[e + 1]);
            }
            const int off = tc::kmaj_off(nu, 4 * g, 128);
            *reinterpret_cast<float4*>(A1h + off) = h1;
            *reinterpret_cast<float4*>(A1l + off) = l1;
            *reinterpret_cast<float4*>(A2h + off) = h2;
            *reinterpret_cast<float4*>(A2l + off) = l2;
        }
    }
};

// node tables of GenS for block (t, s) with direction c: rows pass P = xi_t, Q = xi_s;
// cols pass P = xi_s, Q = xi_t (w negated); reference = the first node of the Q cluster
__device__ void load_node_tables(int32_t t, int32_t s, const double* __restrict__ cd,
                                 const double* __restrict__ nodes, int m, bool rows_pass, float4* P, float4* Q) {
    const int mm = m * m, k = mm * m;
    const int32_t cp = rows_pass ? t : s, cq = rows_pass ? s : t;
    const double sg = rows_pass ? 1.0 : -1.0;
    const double* np_ = nodes + (int64_t)cp * 3 * m;
    const double* nq_ = nodes + (int64_t)cq * 3 * m;
    const double rx = nq_[0], ry = nq_[m], rz = nq_[2 * m];
    // P: 256 entries (two M tiles of 128 rows), zero past k; Q: k entries
    for (int idx = threadIdx.x; idx < 256 + k; idx += blockDim.x) {
        const bool isp = idx < 256;
        const int nu = isp ? idx : idx - 256;
        const double* nn = isp ? np_ : nq_;
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (nu < k) {
            const int ix = nu % m, iy = (nu / m) % m, iz = nu / mm;
            const double x = nn[ix] - rx, y = nn[m + iy] - ry, z = nn[2 * m + iz] - rz;
            v = make_float4((float)x, (float)y, (float)z, (float)(sg * ((x * cd[0] + y * cd[1]) + z * cd[2])));
        }
        if (isp) P[nu] = v;
        else Q[nu] = v;
    }
    __syncthreads();
}

// A[a][mu] = X[a][mu] for rows a < rows of a row-major matrix X (pitch ld), else 0
template <int NT>
struct GenRowsA {
    const cx<float>* X;
    int rows, ld, kmax;
    static constexpr int IT = 128 * TcTile<NT>::KC / kThreads;
    struct Regs {
        cx<float> v[IT];
    };
    __device__ void load(int mu0, Regs& r) const {
#pragma unroll
        for (int it = 0; it < IT; ++it) {   // all loads of the chunk in flight together
            const int idx = threadIdx.x + it * kThreads, core = idx >> 5, w = idx & 31;
            const int a = (core & 15) * 8 + (w >> 2), mu = mu0 + (core >> 4) * 4 + (w & 3);
            r.v[it] = (a < rows && mu < kmax) ? X[(int64_t)a * ld + mu] : zero<float>();
        }
    }
    __device__ void operator()(int, const Regs& r, float* A1h, float* A1l, float* A2h, float* A2l) const {
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int idx = threadIdx.x + it * kThreads;
            tc::split_tf32(r.v[it].x, A1h[idx], A1l[idx]);
            tc::split_tf32(r.v[it].y, A2h[idx], A2l[idx]);
        }
    }
};

// B from the rows of R (row-major, pitch k): B1[i] = Re R_i, B1[i+RP] = Im R_i,
// B2[i] = s Im R_i, B2[i+RP] = -s Re R_i with s = +1 (for conj(S) R^T) or -1 (for S^T R^T)
template <int NT>
struct GenRowsB {
    const cx<float>* Rm;
    int ro, k;
    float s;
    static constexpr int IT = TcTile<NT>::RP * TcTile<NT>::KC / kThreads;
    struct Regs {
        cx<float> rv[IT];
    };
    __device__ void load(int mu0, Regs& r) const {
        constexpr int RP = TcTile<NT>::RP;
#pragma unroll
        for (int it = 0; it < IT; ++it) {   // all loads of the chunk in flight together
            const int idx = threadIdx.x + it * kThreads, core = idx >> 5, w = idx & 31;
            const int i = (core % (RP / 8)) * 8 + (w >> 2), mu = mu0 + (core / (RP / 8)) * 4 + (w & 3);
            r.rv[it] = (i < ro && mu < k) ? Rm[(int64_t)i * k + mu] : zero<float>();
        }
    }
    __device__ void operator()(int, const Regs& regs, float* B1h, float* B1l, float* B2h, float* B2l) const {
        constexpr int RP = TcTile<NT>::RP;
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int idx = threadIdx.x + it * kThreads, core = idx >> 5, w = idx & 31;
            const int i = (core % (RP / 8)) * 8 + (w >> 2), kk = (core / (RP / 8)) * 4 + (w & 3);
            const cx<float> r = regs.rv[it];
            const int o0 = tc::kmaj_off_pad(i, kk, NT), o1 = tc::kmaj_off_pad(i + RP, kk, NT);
            tc::split_tf32(r.x, B1h[o0], B1l[o0]);
            tc::split_tf32(r.y, B1h[o1], B1l[o1]);
            tc::split_tf32(s * r.y, B2h[o0], B2l[o0]);
            tc::split_tf32(-s * r.x, B2h[o1], B2l[o1]);
        }
    }
};

// B from the TMEM tile D1 (rows nu, real parts in columns [0, RP), imaginary in [RP, NT)):
//   conj_d = true  (X conj(D1), X = A1 + i A2):
//     B1[j] = Re D1[.][j], B1[j+RP] = -Im D1[.][j], B2[j] = Im D1[.][j], B2[j+RP] = Re D1[.][j];
//   conj_d = false (conj(X) D1):
//     B1[j] = Re D1[.][j], B1[j+RP] =  Im D1[.][j], B2[j] = Im D1[.][j], B2[j+RP] = -Re D1[.][j].
// The rows nu of a chunk live in TMEM lanes that only warps (chunk quarter) and
// (quarter + 4) may read; each of the two reads half of the columns j.
template <int NT>
struct GenFromTmem {
    uint32_t d1;   // TMEM address of D1 (lane 0, first column); rows nu >= 128 in the next NT columns
    int ro;
    bool conj_d;
    struct Regs {};
    __device__ void load(int, Regs&) const {}
    __device__ void operator()(int mu0, const Regs&, float* B1h, float* B1l, float* B2h, float* B2l) const {
        constexpr int KC = TcTile<NT>::KC, RP = TcTile<NT>::RP;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int z = mu0 >> 7;                 // M tile of D1 holding rows mu0 ... (KC divides 128)
        const int q = (mu0 & 127) >> 5;         // TMEM lane quarter of this chunk (KC <= 32)
        if ((warp & 3) != q) return;
        const int sub = lane - (mu0 & 31);      // row of the chunk held by this lane
        const uint32_t trow = d1 + (uint32_t)(z * NT) + ((uint32_t)(32 * q) << 16);
        const int half = warp >> 2;
        for (int c0 = half * (RP / 2); c0 < (half + 1) * (RP / 2); c0 += 16) {
            float re[16], im[16];
            tc::tmem_ld16(trow + (uint32_t)c0, re);
            tc::tmem_ld16(trow + (uint32_t)(c0 + RP), im);
            if (sub < 0 || sub >= KC) continue;   // lanes of the quarter outside this chunk
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const int j = c0 + jj;
                const float dr = j < ro ? re[jj] : 0.0f, di = j < ro ? im[jj] : 0.0f;
                const int o0 = tc::kmaj_off_pad(j, sub, NT), o1 = tc::kmaj_off_pad(j + RP, sub, NT);
                tc::split_tf32(dr, B1h[o0], B1l[o0]);
                tc::split_tf32(conj_d ? -di : di, B1h[o1], B1l[o1]);
                tc::split_tf32(di, B2h[o0], B2l[o0]);
                tc::split_tf32(conj_d ? dr : -dr, B2h[o1], B2l[o1]);
            }
        }
    }
};

// Tensor-core form of one block task (both passes; see the comment of k_stack_blocks).
// Rows pass: D1 = (R_s S_b^*)^T, then K_b = R_t conj(D1); |G_b|_F = |K_b|_F; the stack rows
// are written once, scaled: w K_b^* for a leaf row cluster, w R_s S_b^* otherwise.  Cols
// pass: (R_t S_b)^T, scaled.  An MMA tile has M = 128 rows, so k <= 256 takes nz = 1 or 2
// tiles of rows nu of D1 (TMEM columns [z NT, (z + 1) NT)) and of rows a of K_b (columns
// [(nz + y) NT, ...)); the CTA holds 2 nz NT TMEM columns.
template <int NT>
__device__ void stack_blocks_tc(const BlockRowTask& tk, bool rows_pass, const float4* Ptab, const float4* Qtab,
                                float kappa, int k,
                                const cx<float>* Ro, int ro, const cx<float>* __restrict__ R,
                                const int64_t* __restrict__ roff, const int32_t* __restrict__ rrows, double* bnorm,
                                cx<float>* out, cx<float>* Kst, float* tcbuf, uint64_t* mbar, uint32_t* tmem_slot,
                                float* red, unsigned* err) {
    constexpr int RP = TcTile<NT>::RP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3, half = warp >> 2;
    const int nz = k > 128 ? 2 : 1;
    const uint32_t ncols = (uint32_t)(2 * nz * NT);
    TcState st;
    tc_begin<NT>(st, tcbuf, mbar, tmem_slot, ncols);
    const uint32_t tq = st.tmem + ((uint32_t)(32 * q) << 16);   // this warp's lane quarter
    const bool kmode = !rows_pass && tk.own_leaf == 2;   // column stack rows w K_b, recomputed
    // D1 = (R_o S^*)^T (sign +1) or (R_o S)^T (cols pass, sign -1), tile by tile
    const float sgn = (!rows_pass && !kmode) ? -1.0f : 1.0f;
    for (int z = 0; z < nz; ++z)
        tc_product<NT>(st, (uint32_t)(z * NT), k, GenS<NT>{Ptab + 128 * z, Qtab, k, kappa, k - 128 * z},
                       GenRowsB<NT>{Ro, ro, k, sgn});
    if (!rows_pass && !kmode) {
        const float sc_ = bnorm[tk.b] > 0.0 ? float(1.0 / bnorm[tk.b]) : 0.0f;
        if (st.ok) {
            for (int z = 0; z < nz; ++z) {
                const int row = 128 * z + 32 * q + lane;   // nu
                for (int c0 = half * (RP / 2); c0 < (half + 1) * (RP / 2) && c0 < ro; c0 += 16) {
                    float re[16], im[16];
                    tc::tmem_ld16(tq + (uint32_t)(z * NT + c0), re);
                    tc::tmem_ld16(tq + (uint32_t)(z * NT + c0 + RP), im);
                    if (row < k)
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < ro) out[(int64_t)(c0 + j) * k + row] = cx<float>{sc_ * re[j], sc_ * im[j]};
                }
            }
        }
        tc_end<NT>(st, err, ncols);
        return;
    }
    const int rt = rrows[tk.own];
    const int ny = rt > 128 ? 2 : 1;   // rt <= k <= 128 nz
    const cx<float>* Rt = R + roff[tk.own];
    cx<float>* Kb = (Kst && !kmode) ? Kst + tk.koff : nullptr;   // stored only if there is a store
    for (int y = 0; y < ny; ++y)
        tc_product<NT>(st, (uint32_t)((nz + y) * NT), k, GenRowsA<NT>{Rt + (int64_t)128 * y * k, rt - 128 * y, k, k},
                       GenFromTmem<NT>{st.tmem, ro, true});
    // K_b (rows a = TMEM lanes of tile y, columns j < ro) and |K_b|_F
    float acc = 0.0f;
    if (st.ok) {
        for (int y = 0; y < ny; ++y) {
            const int row = 128 * y + 32 * q + lane;   // a
            for (int c0 = half * (RP / 2); c0 < (half + 1) * (RP / 2) && c0 < ro; c0 += 16) {
                float re[16], im[16];
                tc::tmem_ld16(tq + (uint32_t)((nz + y) * NT + c0), re);
                tc::tmem_ld16(tq + (uint32_t)((nz + y) * NT + c0 + RP), im);
                if (row < rt)
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < ro) {
                            if (Kb) Kb[(int64_t)row * ro + c0 + j] = cx<float>{re[j], im[j]};
                            acc += re[j] * re[j] + im[j] * im[j];
                        }
            }
        }
    }
    const float nrm = sqrtf(block_sum(acc, red));
    if (threadIdx.x == 0 && !kmode) bnorm[tk.b] = (double)nrm;
    const float sc_ = nrm > 0.0f ? 1.0f / nrm : 0.0f;
    if (st.ok) {
        if (kmode || tk.own_leaf) {
            // kmode: w K_b, column-stack row a (< rt), column j (< ro), pitch k;
            // leaf row cluster: w K_b^*, stack row j (< ro), column a (< rt), pitch k
            for (int y = 0; y < ny; ++y) {
                const int row = 128 * y + 32 * q + lane;   // a
                for (int c0 = half * (RP / 2); c0 < (half + 1) * (RP / 2) && c0 < ro; c0 += 16) {
                    float re[16], im[16];
                    tc::tmem_ld16(tq + (uint32_t)((nz + y) * NT + c0), re);
                    tc::tmem_ld16(tq + (uint32_t)((nz + y) * NT + c0 + RP), im);
                    if (row < rt)
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < ro) {
                                const cx<float> v{sc_ * re[j], (kmode ? sc_ : -sc_) * im[j]};
                                if (!isfinite(v.x) || !isfinite(v.y)) raise_err(err, ERR_STACK_NONFINITE);
                                if (kmode) out[(int64_t)row * k + c0 + j] = v;
                                else out[(int64_t)(c0 + j) * k + row] = v;
                            }
                }
            }
        } else {
            // w R_s S_b^*: stack row i (< ro), column nu (< k)
            for (int z = 0; z < nz; ++z) {
                const int row = 128 * z + 32 * q + lane;   // nu
                for (int c0 = half * (RP / 2); c0 < (half + 1) * (RP / 2) && c0 < ro; c0 += 16) {
                    float re[16], im[16];
                    tc::tmem_ld16(tq + (uint32_t)(z * NT + c0), re);
                    tc::tmem_ld16(tq + (uint32_t)(z * NT + c0 + RP), im);
                    if (row < k)
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < ro) {
                                const cx<float> v{sc_ * re[j], sc_ * im[j]};
                                if (!isfinite(v.x) || !isfinite(v.y)) raise_err(err, ERR_STACK_NONFINITE);
                                out[(int64_t)(c0 + j) * k + row] = v;
                            }
                }
            }
        }
    }
    tc_end<NT>(st, err, ncols);
}

// rows pass: R_sc S_b^*, then |G_b|_F = |R_tc S_b R_sc^*|_F, rows scaled by 1/|G_b|.
// cols pass: R_tc S_b / |G_b|.
template <class T, int NT>
__global__ void __launch_bounds__(256, 2) k_stack_blocks(const BlockRowTask* __restrict__ tasks, bool rows_pass,
                               const int32_t* __restrict__ adm_t, const int32_t* __restrict__ adm_s,
                               const int32_t* __restrict__ adm_c, const int32_t* __restrict__ tc_level,
                               const int32_t* __restrict__ dir_off, const double* __restrict__ dirs,
                               const double* __restrict__ nodes, int m, double kappa,
                               const cx<T>* __restrict__ Rv, const cx<T>* __restrict__ Rw,
                               const int64_t* __restrict__ roff, const int32_t* __restrict__ rrows, double* bnorm,
                               cx<T>* stack, cx<T>* Kst, unsigned* err) {
    extern __shared__ unsigned char smraw[];
    __shared__ T red[32];
    const BlockRowTask tk = tasks[blockIdx.x];
    const int k = m * m * m;
    const int32_t t = adm_t[tk.b], s = adm_s[tk.b], c = adm_c[tk.b];
    const double* cd = dirs + 3 * (dir_off[tc_level[t]] + c);
    const int ro = rrows[tk.other];
    // Rv: weights of the row basis V, Rw: of the column basis W (the same array for the
    // single layer).  The "other" pair is a column cluster s in the rows pass and in the
    // recomputed K_b rows, a row cluster t otherwise; the "own" pair is always a row cluster.
    const cx<T>* R = Rv;
    const cx<T>* Ro = ((rows_pass || tk.own_leaf == 2) ? Rw : Rv) + roff[tk.other];
    cx<T>* out = stack + tk.dst;
    if constexpr (NT > 0) {
        // node tables (2 x 128 float4), then the tensor-core operands on a 128-byte boundary
        __shared__ __align__(8) uint64_t tc_mbar[1];
        __shared__ uint32_t tc_tmem;
        float4* Ptab = reinterpret_cast<float4*>(
            (reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
        float4* Qtab = Ptab + 256;
        float* tcbuf = reinterpret_cast<float*>(Qtab + 256);
        load_node_tables(t, s, cd, nodes, m, rows_pass || tk.own_leaf == 2, Ptab, Qtab);
        stack_blocks_tc<NT>(tk, rows_pass, Ptab, Qtab, (float)kappa, k, Ro, ro, R, roff, rrows, bnorm, out, Kst,
                            tcbuf, tc_mbar, &tc_tmem, red, err);
        return;
    }
    const SGen<T> S = load_sgen_tables<T>(t, s, cd, nodes, m, kappa, smraw);
    if (rows_pass) {
        // out[i][nu] = sum_mu R_s[i][mu] conj(S[nu][mu])
        cta_gemm_fit<T>(ro, k, k, Dense<T>{Ro, k, false, false},
                    [&](int mu, int nu) { return conj(S(nu, mu)); },
                    [&](int i, int nu, cx<T> v) { out[(int64_t)i * k + nu] = v; });
        __syncthreads();
        // K_b = R_t S R_s^* = R_t Y with Y[nu][i] = conj(out[i][nu]); |G_b|_F = |K_b|_F
        const int rt = rrows[tk.own];
        const cx<T>* Rt = R + roff[tk.own];
        cx<T>* Kb = Kst + tk.koff;
        T acc = 0;
        T* accp = &acc;
        cta_gemm_fit<T>(rt, ro, k, Dense<T>{Rt, k, false, false}, Dense<T>{out, k, true, true},
                    [=](int i, int j, cx<T> v) {
                        *accp += abs2(v);
                        Kb[(int64_t)i * ro + j] = v;
                    });
        T nrm2 = block_sum(acc, red);
        T nrm = sqrt(nrm2);
        if (threadIdx.x == 0) bnorm[tk.b] = (double)nrm;
        T sc_ = nrm > T(0) ? T(1) / nrm : T(0);
        __syncthreads();
        if (tk.own_leaf) {
            // rows projected onto the leaf's orthonormal basis: w K_b^*  (ro x rt, pitch k)
            for (int idx = threadIdx.x; idx < ro * rt; idx += blockDim.x) {
                const int i = idx / rt, j = idx - i * rt;
                cx<T> v = sc_ * conj(Kb[(int64_t)j * ro + i]);
                if (!isfinite(v.x) || !isfinite(v.y)) raise_err(err, ERR_STACK_NONFINITE);
                out[(int64_t)i * k + j] = v;
            }
        } else {
            for (int idx = threadIdx.x; idx < ro * k; idx += blockDim.x) {
                cx<T> v = sc_ * out[idx];
                if (!isfinite(v.x) || !isfinite(v.y)) raise_err(err, ERR_STACK_NONFINITE);
                out[idx] = v;
            }
        }
    } else {
        const T sc_ = bnorm[tk.b] > 0.0 ? T(1.0 / bnorm[tk.b]) : T(0);
        // out[i][nu] = sum_mu R_t[i][mu] S[mu][nu] / |G_b|
        cta_gemm_fit<T>(ro, k, k, Dense<T>{Ro, k, false, false},
                    [&](int mu, int nu) { return S(mu, nu); },
                    [&](int i, int nu, cx<T> v) { out[(int64_t)i * k + nu] = sc_ * v; });
    }
}

struct KronTask {
    int64_t src;       // element offset of the first input row
    int64_t fac;       // element offset of the 3 m x m factors
    int64_t dst;       // element offset of the first output row
    int32_t rows;
    int32_t adjoint;
};

// out rows = in rows * E (or * E^*), computed in TC, stored as TO
template <class TI, class TF, class TC, class TO>
__global__ void k_kron(const KronTask* __restrict__ tasks, int m, const cx<TI>* __restrict__ in,
                       const cx<TF>* __restrict__ fac, cx<TO>* out) {
    extern __shared__ unsigned char smraw[];
    cx<TC>* buf = reinterpret_cast<cx<TC>*>(smraw);
    const KronTask tk = tasks[blockIdx.x];
    const int k = m * m * m;
    cx<TC>* F = buf + 2 * k;
    for (int i = threadIdx.x; i < 3 * m * m; i += blockDim.x) {
        cx<TF> f = fac[tk.fac + i];
        F[i] = cx<TC>{TC(f.x), TC(f.y)};
    }
    __syncthreads();
    const cx<TI>* X = in + tk.src;
    cx<TO>* O = out + tk.dst;
    kron_apply<TC>(tk.rows, m, F, tk.adjoint != 0,
                   [&](int r, int v) {
                       cx<TI> x = X[(int64_t)r * k + v];
                       return cx<TC>{TC(x.x), TC(x.y)};
                   },
                   [&](int r, int v, cx<TC> val) { O[(int64_t)r * k + v] = cx<TO>{TO(val.x), TO(val.y)}; },
                   buf);
}

// ----------------------------------------------------------------------------- TSQR

struct QRTask {
    int64_t src;       // element offset of the first stacked row
    int64_t dst;       // element offset of the output rows (compact, ncols per row)
    int32_t nrows;
    int32_t rout;      // min(nrows, ncols) rows written to dst
    int32_t ncols;     // columns of this task (<= the launch's k)
    int32_t ld;        // row pitch of the source rows
};

constexpr int kQRNB = 8;   // panel width of the blocked Householder update

// FP32 one-sided Jacobi of the mixed form: stop when every pair has |g| <= tol sqrt(a b)
// (a few units of FP32 rounding over rows of ~100 entries), at most this many sweeps.
constexpr float kJacobiTolF32 = 4e-6f;
constexpr int kJacobiSweepsF32 = 16;

// R-factor of the stacked rows: R scratch (k x k, TQ) per CTA, chunks of 32*RPL rows.
// Reads TSrc, writes the rout leading rows of R as TDst.
template <class TSrc, class TQ, class TDst, int RPL>
__global__ void __launch_bounds__(256) k_tsqr(const QRTask* __restrict__ tasks, int k,
                                              const cx<TSrc>* __restrict__ src, cx<TQ>* scratch,
                                              cx<TDst>* dst, unsigned* err) {
    extern __shared__ unsigned char smraw[];
    constexpr int H = 32 * RPL, LDW = H + 1;
    cx<TQ>* W = reinterpret_cast<cx<TQ>*>(smraw);
    cx<TQ>* s_Wm = W + (int64_t)k * LDW;
    cx<TQ>* s_T = s_Wm + (int64_t)kQRNB * k;
    cx<TQ>* s_G = s_T + kQRNB * kQRNB;
    cx<TQ>* s_tau = s_G + kQRNB * kQRNB;
    int* s_skip = reinterpret_cast<int*>(s_tau + kQRNB);
    const QRTask tk = tasks[blockIdx.x];
    const int nc = tk.ncols;
    cx<TQ>* R = scratch + (int64_t)blockIdx.x * k * k;
    for (int idx = threadIdx.x; idx < nc * nc; idx += blockDim.x) R[idx] = zero<TQ>();
    __syncthreads();
    const cx<TSrc>* S = src + tk.src;
    for (int r0 = 0; r0 < tk.nrows; r0 += H) {
        const int h = min(H, tk.nrows - r0);
        for (int idx = threadIdx.x; idx < H * nc; idx += blockDim.x) {
            const int i = idx / nc, l = idx - i * nc;     // row-major read, column-major store
            cx<TQ> v = zero<TQ>();
            if (i < h) {
                cx<TSrc> u = S[(int64_t)(r0 + i) * tk.ld + l];
                if (!isfinite(u.x) || !isfinite(u.y)) raise_err(err, ERR_TSQR_INPUT);
                v = cx<TQ>{TQ(u.x), TQ(u.y)};
            }
            W[(int64_t)l * LDW + i] = v;
        }
        __syncthreads();
        tsqr_chunk<TQ, RPL, kQRNB>(nc, R, W, s_tau, s_skip, s_T, s_G, s_Wm);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < tk.rout * nc; idx += blockDim.x) {
        cx<TQ> v = R[idx];
        if (!isfinite(v.x) || !isfinite(v.y)) raise_err(err, ERR_TSQR_NONFINITE);
        dst[tk.dst + idx] = cx<TDst>{TDst(v.x), TDst(v.y)};
    }
}

// R-factor of the stacked rows for FP32 stacks of at most 256 / TPC columns, column
// parallel: the TPC consecutive threads of column l hold rows sub*RT + i (i < RT) of the
// current chunk of H = TPC*RT rows in registers.  Column j's owners build its reflector
// (xLARFG convention, scaled column as in tsqr_chunk) and post it in shared memory; after
// one block barrier every later column applies it with a dot product inside its threads
// and a log2(TPC)-step shuffle.  Row j of R (global scratch, pitch ncols) only meets
// column l's owners, so R needs no further synchronisation; the next row is fetched one
// step ahead.
// Reductions over the TPC lanes of one column.  They run inside branches that only that
// column's lanes take, so the shuffle mask names exactly those lanes (all of which
// execute the same shuffles), never the whole warp.
template <int TPC>
__device__ __forceinline__ unsigned group_mask() {
    const unsigned lane = threadIdx.x & 31u;
    return (TPC == 32 ? 0xffffffffu : ((1u << TPC) - 1u)) << (lane & ~(unsigned)(TPC - 1));
}
template <int TPC>
__device__ __forceinline__ float group_max(float v) {
    const unsigned mask = group_mask<TPC>();
#pragma unroll
    for (int o = 1; o < TPC; o <<= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o));
    return v;
}
template <int TPC>
__device__ __forceinline__ float group_sum_r(float v) {
    const unsigned mask = group_mask<TPC>();
#pragma unroll
    for (int o = 1; o < TPC; o <<= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}
template <int TPC>
__device__ __forceinline__ cx<float> group_sum(cx<float> v) {
    const unsigned mask = group_mask<TPC>();
#pragma unroll
    for (int o = 1; o < TPC; o <<= 1) v = cx<float>{v.x + __shfl_xor_sync(mask, v.x, o), v.y + __shfl_xor_sync(mask, v.y, o)};
    return v;
}

template <int TPC, int RT, class TSrc, class TDst>
__global__ void __launch_bounds__(256, 3) k_tsqr_cols(const QRTask* __restrict__ tasks, int kl,
                                                      const cx<TSrc>* __restrict__ src, cx<float>* scratch,
                                                      cx<TDst>* dst, unsigned* err) {
    static_assert(RT % 4 == 0, "rows per thread");
    constexpr int H = TPC * RT;
    constexpr int SL = RT + 2;   // slice pitch: one spare 16-byte word staggers the banks
    __shared__ __align__(16) cx<float> vbuf[2][TPC * SL];
    __shared__ cx<float> taub[2];
    const QRTask tk = tasks[blockIdx.x];
    const int nc = tk.ncols;
    const int col = threadIdx.x / TPC, sub = threadIdx.x % TPC;
    const int warp = threadIdx.x >> 5;
    const bool mine = col < nc;
    cx<float>* R = scratch + (int64_t)blockIdx.x * kl * kl;
    for (int idx = threadIdx.x; idx < nc * nc; idx += blockDim.x) R[idx] = zero<float>();
    __syncthreads();
    const cx<TSrc>* S = src + tk.src;
    bool bad = false;
    cx<float> w[RT];   // rows sub*RT + i of this column
    for (int r0 = 0; r0 < tk.nrows; r0 += H) {
        const int h = min(H, tk.nrows - r0);
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            const int row = sub * RT + i;
            cx<float> v = zero<float>();
            if (mine && row < h) {
                const cx<TSrc> u = S[(int64_t)(r0 + row) * tk.ld + col];
                bad |= !isfinite(u.x) || !isfinite(u.y);
                v = cx<float>{float(u.x), float(u.y)};
            }
            w[i] = v;
        }
        cx<float> rj = mine ? R[col] : zero<float>();   // R[j][col] for j = 0
        // Step j involves the warps that hold a column >= j: [fa, nwv) with fa the warp of
        // column j.  A warp whose columns are all < j is done with this chunk and leaves the
        // loop; the others meet at named barrier 1 with exactly that many threads.
        const int nwv = (nc * TPC + 31) / 32;
        for (int j = 0; j < nc && warp < nwv; ++j) {
            const int fa = (j * TPC) / 32;
            if (warp < fa) break;
            const int b = j & 1;
            const cx<float> rnext = (mine && j + 1 < nc) ? R[(j + 1) * nc + col] : zero<float>();
            float4* vq = reinterpret_cast<float4*>(&vbuf[b][sub * SL]);
            if (col == j) {
                // reflector of column j; uniform over the TPC owners.  Four partial
                // maxima / sums keep the dependency chains short.
                float m4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int i = 0; i < RT; ++i) m4[i & 3] = fmaxf(m4[i & 3], fmaxf(fabsf(w[i].x), fabsf(w[i].y)));
                const float xmax = group_max<TPC>(fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3])));
                if (xmax >= 1.17549435e-38f) {
                    const float amax = fmaxf(xmax, fmaxf(fabsf(rj.x), fabsf(rj.y)));
                    const float inv = 1.0f / amax;
                    float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                    for (int i = 0; i < RT; ++i) s4[i & 3] += abs2(inv * w[i]);
                    const float xn2 = group_sum_r<TPC>((s4[0] + s4[1]) + (s4[2] + s4[3]));
                    const cx<float> als = inv * rj;
                    const float betas = -copysignf(sqrtf(abs2(als) + xn2), als.x);   // beta / amax
                    const float rb = 1.0f / betas;
                    const cx<float> tauc = mk<float>((betas - als.x) * rb, als.y * rb);
                    const cx<float> d = mk<float>(als.x - betas, als.y);
                    const float dn = inv / abs2(d);
                    const cx<float> sc = mk<float>(d.x * dn, -d.y * dn);   // 1 / (alpha - beta)
#pragma unroll
                    for (int i = 0; i < RT; i += 2) {
                        const cx<float> a0 = w[i] * sc, a1 = w[i + 1] * sc;
                        vq[i / 2] = make_float4(a0.x, a0.y, a1.x, a1.y);
                    }
                    if (sub == 0) {
                        R[j * nc + j] = mk<float>(betas * amax, 0.0f);
                        taub[b] = tauc;
                    }
                } else {   // numerically zero column: identity reflector
#pragma unroll
                    for (int i = 0; i < RT; i += 2) vq[i / 2] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (sub == 0) taub[b] = zero<float>();
                }
            }
            asm volatile("bar.sync 1, %0;" :: "r"(32 * (nwv - fa)) : "memory");
            if (mine && col > j) {
                const cx<float> tauc = taub[b];
                cx<float> d4[4] = {zero<float>(), zero<float>(), zero<float>(), zero<float>()};
#pragma unroll
                for (int i = 0; i < RT; i += 2) {
                    const float4 q = vq[i / 2];
                    fma_cjx(d4[i & 3], cx<float>{q.x, q.y}, w[i]);
                    fma_cjx(d4[(i + 1) & 3], cx<float>{q.z, q.w}, w[i + 1]);
                }
                const cx<float> sdot = group_sum<TPC>((d4[0] + d4[1]) + (d4[2] + d4[3]));
                const cx<float> tw = tauc * (rj + sdot);
                // read the reflector again rather than keep RT more values in registers
                asm volatile("" ::: "memory");
#pragma unroll
                for (int i = 0; i < RT; i += 2) {
                    const float4 q = vq[i / 2];
                    w[i] = w[i] - cx<float>{q.x, q.y} * tw;
                    w[i + 1] = w[i + 1] - cx<float>{q.z, q.w} * tw;
                }
                if (sub == 0) R[j * nc + col] = rj - tw;
            }
            rj = rnext;
        }
        __syncthreads();   // the next chunk's first reflector reuses vbuf[0]
    }
    if (bad) raise_err(err, ERR_TSQR_INPUT);
    __syncthreads();
    for (int idx = threadIdx.x; idx < tk.rout * nc; idx += blockDim.x) {
        const int i = idx / nc, l = idx - i * nc;
        const cx<float> v = l >= i ? R[idx] : zero<float>();
        if (!isfinite(v.x) || !isfinite(v.y)) raise_err(err, ERR_TSQR_NONFINITE);
        dst[tk.dst + idx] = cx<TDst>{TDst(v.x), TDst(v.y)};
    }
}

// A stack with no more rows than columns is its own R factor: R = Z gives R^* R = Z^* Z
// exactly, which is all the method uses of R.  (Merging such a stack into a zero R by
// Householder reflections and keeping min(rows, cols) rows would drop the rounding noise
// that the reflections leave in the further rows; with ill-conditioned leading columns
// that noise is amplified far above u |Z|.)  One CTA per stack, rows converted to TDst.
template <class TSrc, class TDst>
__global__ void k_copy_rows(const QRTask* __restrict__ tasks, const cx<TSrc>* __restrict__ src,
                            cx<TDst>* __restrict__ dst, unsigned* err) {
    const QRTask tk = tasks[blockIdx.x];
    bool bad = false;
    for (int idx = threadIdx.x; idx < tk.rout * tk.ncols; idx += blockDim.x) {
        const int i = idx / tk.ncols, l = idx - i * tk.ncols;
        const cx<TSrc> u = i < tk.nrows ? src[tk.src + (int64_t)i * tk.ld + l] : zero<TSrc>();
        bad |= !isfinite(u.x) || !isfinite(u.y);
        dst[tk.dst + idx] = cx<TDst>{TDst(u.x), TDst(u.y)};
    }
    if (bad) raise_err(err, ERR_TSQR_INPUT);
}

// ----------------------------------------------------------------------------- FP64 Cholesky QR

// R-factor of a stacked matrix Z (H x c) in FP64 through its Gram matrix: G = Z^* Z
// accumulated in FP64 (Hermitian, upper tiles only), then a pivoted Cholesky G = R^* R
// with R (rout x c) dense rows: row j holds the j-th pivot's entries in the original
// column order.  Only R^* R = Z^* Z enters the method (the stacks of Eq. basis_weights_def
// and Eq. recomp_weight_full and the truncation use R through products whose Gram is
// that of Z), so R may differ from a Householder R by a unitary left factor.  The Gram
// has absolute rounding error ~ u_64 |Z|^2, which moves the squared singular values that
// the rank rule sums by the same absolute amount, far below eps^2 |Z|^2.

// One tile of the Gram matrix: columns [i0, i0 + TB) x [j0, j0 + TB), i0 <= j0, over the
// stacked rows [r0, r1).
struct GramItem {
    int64_t src;              // element offset of the stack's first row
    int64_t out;              // cx<double> offset of this partial tile (TB x TB, row-major)
    int32_t ld, ncols, r0, r1;
    int32_t i0, j0;
    int32_t half;             // k_gram_slices: the real (0) or imaginary (1) parts of columns j0..
    int32_t narrow;           // k_gram_slices: a stack of at most 32 columns, one CTA per tile
    int64_t cmax;             // k_gram_slices: offset of the row group's column maxima (2 ncols)
};

// Column maxima of a stack's row group for k_gram_slices: max |Re z_c| at cmax[2 c] and
// max |Im z_c| at cmax[2 c + 1] over rows r0 .. r1 - 1 (FP32 bit patterns, combined by
// atomicMax over the slices of a group; the buffer starts at zero).
struct ColMaxTask {
    int64_t src, cmax;
    int32_t ld, ncols, r0, r1;
};

// max |Re|, |Im| of one column over rows r, r + step, ... < r1 (eight loads in flight)
__device__ __forceinline__ void colmax_rows(const cx<float>* S, int64_t ld, int r, int r1, int step, uint32_t* out,
                                            unsigned* err) {
    float mr = 0.0f, mi = 0.0f;
    bool bad = false;
    for (; r + 7 * step < r1; r += 8 * step) {
        cx<float> u[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) u[t] = S[(int64_t)(r + t * step) * ld];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            bad |= !isfinite(u[t].x) || !isfinite(u[t].y);
            mr = fmaxf(mr, fabsf(u[t].x));
            mi = fmaxf(mi, fabsf(u[t].y));
        }
    }
    for (; r < r1; r += step) {
        const cx<float> u = S[(int64_t)r * ld];
        bad |= !isfinite(u.x) || !isfinite(u.y);
        mr = fmaxf(mr, fabsf(u.x));
        mi = fmaxf(mi, fabsf(u.y));
    }
    if (bad) raise_err(err, ERR_TSQR_INPUT);
    atomicMax(&out[0], __float_as_uint(mr));   // non-negative floats order as their bit patterns
    atomicMax(&out[1], __float_as_uint(mi));
}

__global__ void __launch_bounds__(256) k_gram_colmax(const ColMaxTask* __restrict__ tasks,
                                                     const cx<float>* __restrict__ src, uint32_t* cmax,
                                                     unsigned* err) {
    const ColMaxTask tk = tasks[blockIdx.x];
    const int C = tk.ncols, t = threadIdx.x, nt = blockDim.x;
    const cx<float>* S = src + tk.src;
    if (C <= nt) {   // nt / C threads per column, consecutive threads on consecutive columns
        const int tpc = nt / C, c = t % C, ph = t / C;
        if (ph < tpc) colmax_rows(S + c, tk.ld, tk.r0 + ph, tk.r1, tpc, cmax + tk.cmax + 2 * c, err);
    } else {
        for (int c = t; c < C; c += nt) colmax_rows(S + c, tk.ld, tk.r0, tk.r1, 1, cmax + tk.cmax + 2 * c, err);
    }
}

// TB = 16 * BS: each of up to 256 threads accumulates a BS x BS block of the tile in
// FP64 registers; on a diagonal tile only the blocks on or above the diagonal are
// computed, handed out to consecutive threads so that whole warps of the rest stay idle.
// Rows are staged RC at a time in shared memory, converted to FP64 once.
template <int BS, class TSrc>
__global__ void __launch_bounds__(256) k_gram64(const GramItem* __restrict__ items, const cx<TSrc>* __restrict__ src,
                                                cx<double>* __restrict__ part, unsigned* err) {
    // rows per staged chunk: 16 for 64-column tiles (1024 FP64 FMA per thread per chunk),
    // 32 for 32-column tiles, whose threads do a quarter of that per row
    constexpr int TB = 16 * BS, RC = BS >= 4 ? 16 : 32;
    __shared__ cx<double> sa[RC][TB], sb[RC][TB];
    const GramItem it = items[blockIdx.x];
    const bool diag = it.i0 == it.j0;
    const int nbi = min(16, (it.ncols - it.i0 + BS - 1) / BS);
    const int nbj = min(16, (it.ncols - it.j0 + BS - 1) / BS);
    int bi = -1, bj = -1;
    {
        int t = threadIdx.x;
        if (diag) {
            for (int r = 0; r < nbi; ++r) {   // block row r holds nbi - r blocks
                const int cnt = nbi - r;
                if (t < cnt) {
                    bi = r;
                    bj = r + t;
                    break;
                }
                t -= cnt;
            }
        } else if (t < nbi * nbj) {
            bi = t / nbj;
            bj = t - bi * nbj;
        }
    }
    const bool active = bi >= 0;
    cx<double> acc[BS][BS];
#pragma unroll
    for (int p = 0; p < BS; ++p)
#pragma unroll
        for (int q = 0; q < BS; ++q) acc[p][q] = zero<double>();
    const cx<TSrc>* S = src + it.src;
    bool bad = false;
    for (int h0 = it.r0; h0 < it.r1; h0 += RC) {
        const int hh = min(RC, it.r1 - h0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < RC * TB; idx += blockDim.x) {
            const int r = idx / TB, c = idx - r * TB;
            cx<double> a = zero<double>(), b = zero<double>();
            if (r < hh) {
                const int64_t row = (int64_t)(h0 + r) * it.ld;
                if (it.i0 + c < it.ncols) {
                    const cx<TSrc> u = S[row + it.i0 + c];
                    bad |= !isfinite(u.x) || !isfinite(u.y);
                    a = cx<double>{double(u.x), double(u.y)};
                }
                if (!diag && it.j0 + c < it.ncols) {
                    const cx<TSrc> u = S[row + it.j0 + c];
                    bad |= !isfinite(u.x) || !isfinite(u.y);
                    b = cx<double>{double(u.x), double(u.y)};
                }
            }
            sa[r][c] = a;
            if (!diag) sb[r][c] = b;
        }
        __syncthreads();
        if (active) {
            const cx<double>(*B)[TB] = diag ? sa : sb;
            for (int r = 0; r < hh; ++r) {
                cx<double> a[BS], b[BS];
#pragma unroll
                for (int q = 0; q < BS; ++q) {
                    a[q] = sa[r][bi * BS + q];
                    b[q] = B[r][bj * BS + q];
                }
#pragma unroll
                for (int p = 0; p < BS; ++p)
#pragma unroll
                    for (int q = 0; q < BS; ++q) fma_cjx(acc[p][q], a[p], b[q]);
            }
        }
    }
    if (bad) raise_err(err, ERR_TSQR_INPUT);
    if (active) {
        cx<double>* O = part + it.out;
#pragma unroll
        for (int p = 0; p < BS; ++p)
#pragma unroll
            for (int q = 0; q < BS; ++q) O[(bi * BS + p) * TB + bj * BS + q] = acc[p][q];
    }
}

// ----------------------------------------------------------------------------- Gram from integer slices

// The Gram tile G = Z_I^* Z_J of an FP32 stack (I, J: 64 complex columns each) from exact
// integer products on the BF16 tensor cores.  Each real column m of the tile (the real and
// the imaginary parts of a complex column are two real columns) is scaled by 2^-e_m, e_m the
// exponent of its largest magnitude over the row group, and written as 8 signed base-64
// digits, x 2^-e_m = sum_i d_i 2^(1 - 6 i) + rest, |d_i| <= 32, |rest| <= 2^-48: each digit is
// the remainder rounded to the next grid 2^(-6 i), so every step is exact in FP32 and every
// digit (kept at its weight) exact in BF16.  A dot product of two columns is then
// sum_{i,j} (d_i . d'_j) 2^(2 - 6(i+j)); the digit products with one i + j = g share that grid
// and are summed in one FP32 TMEM accumulator, whose partial sums are integer multiples of it
// of magnitude at most 8 * 32 * 32 * rows <= 2^24 units for rows <= 2048, so the tensor cores
// add them exactly.  Products with i + j > 9 are dropped;
// with the rests this leaves an error of at most about 2^-43 max|z_m| max|z_n| per row (an FP64
// accumulation: 2^-53 |z_m| |z_n|), far below the FP32 rounding of the stack's own entries.
//
// The real product is split by the column part of J: a CTA with half = 0 forms D = Y_I^T Re Z_J
// and one with half = 1 forms D = Y_I^T Im Z_J, Y_I = [Re Z_I, Im Z_I] (M = 128 rows), and each
// writes one complex partial tile: half 0 (Re G, Im G) = (D_top, -D_bottom), half 1
// (D_bottom, D_top).  The 8 group accumulators (64 columns each) take all 512 TMEM columns (one
// CTA per SM).  The digits of J's part are stored digit after digit as one operand of 512 rows,
// so one MMA multiplies digit i of Y_I by up to four consecutive digits j of Z_J (N <= 256) and
// writes the consecutive groups i + j: 14 MMAs per 16 rows, each accumulator run starting at a
// TMEM column that is a multiple of its width.  The digits of 32 rows are
// staged per step in two shared-memory buffers; the rows of the next step are loaded into
// registers and the digits of the next step formed while the tensor cores work on the current.
namespace gram_tc {
constexpr int kDigits = 8;
constexpr int kMaxRows = 2048;
constexpr int kSub = 32;
constexpr int kABytes = kDigits * 128 * kSub * 2;   // digits of Y_I: per digit 128 rows x kSub
constexpr int kBBytes = kDigits * 64 * kSub * 2;    // digits of one part of Z_J: 512 rows x kSub
constexpr int kHeader = 2048;
constexpr size_t kSmemBytes = 1024 + kHeader + 2 * (size_t)(kABytes + kBBytes);   // 1024: alignment

// two FP32 lanes at once (Blackwell packed arithmetic): rows t and t + 1 of a column
__device__ __forceinline__ uint64_t fadd2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fsub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t pack2(float a, float b) {
    return (uint64_t)__float_as_uint(a) | ((uint64_t)__float_as_uint(b) << 32);
}

// The digits of 8 consecutive rows (y = x 2^(5 - e), |y| <= 32) of one real column, each at its
// own weight: digit d is y's remainder rounded to the grid 2^(-6 d) (adding and subtracting
// 1.5 * 2^(23 - 6 d) rounds to that grid; the remainder then loses the digit exactly), so
// digit d = s 2^(-6 d) with an integer |s| <= 32 and y = sum of the digits + rest, |rest| <=
// 2^-43.  Stored as one 16-byte core-matrix row per digit (K-major layouts, see tcgen05.cuh):
// at row r of digit d's 128-row block of A (a != nullptr) and at row 64 d + rb of the 512-row
// B (b != nullptr).
__device__ __forceinline__ void store_digits(float (&y)[8], unsigned char* a, int r, unsigned char* b, int rb, int q) {
    const int offa = tc::kmaj_off16(r, 8 * q, 128) * 2;
    uint64_t v2[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) v2[t] = pack2(y[2 * t], y[2 * t + 1]);
#pragma unroll
    for (int d = 0; d < kDigits; ++d) {
        const float R = 12582912.0f * __int_as_float((127 - 6 * d) << 23);   // 1.5 * 2^(23 - 6 d)
        const uint64_t R2 = pack2(R, R);
        uint32_t w[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint64_t sd = fsub2(fadd2(v2[t], R2), R2);   // the digits of rows 2t, 2t + 1
            v2[t] = fsub2(v2[t], sd);
            // each digit has at most 6 significant bits: its FP32 pattern's low half is zero
            w[t] = __byte_perm((uint32_t)sd, (uint32_t)(sd >> 32), 0x7632);
        }
        const uint4 v{w[0], w[1], w[2], w[3]};
        if (a) *reinterpret_cast<uint4*>(a + d * (128 * kSub * 2) + offa) = v;
        if (b) *reinterpret_cast<uint4*>(b + tc::kmaj_off16(64 * d + rb, 8 * q, 512) * 2) = v;
    }
}

// FP32 -> FP64 with e added to the exponent, by integer operations (f normal or zero)
__device__ __forceinline__ double widen(float f, int e) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t E = (b >> 23) & 0xFFu;
    if (E == 0) return 0.0;
    const uint32_t hi = (b & 0x80000000u) | ((E + 896u + (uint32_t)e) << 20) | ((b >> 3) & 0xFFFFFu);
    return __hiloint2double((int)hi, (int)(b << 29));
}
}  // namespace gram_tc

// 288 threads: warps 0-7 form the digits (and drain the accumulators), warp 8 issues the MMAs.
// Per buffer, `full` counts the 8 producer warps' arrivals and `empty` is signalled by the
// tensor cores (tcgen05.commit) once the MMAs reading it are done; every wait is bounded.
__global__ void __launch_bounds__(288, 1) k_gram_slices(const GramItem* __restrict__ items,
                                                        const cx<float>* __restrict__ src,
                                                        const uint32_t* __restrict__ cmax,
                                                        cx<double>* __restrict__ part, unsigned* err) {
    using namespace gram_tc;
    extern __shared__ unsigned char g_smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(g_smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    uint32_t* colbits = reinterpret_cast<uint32_t*>(base);   // 192: column maxima, then exponents
    int* ex = reinterpret_cast<int*>(base);
    float* scl = reinterpret_cast<float*>(base + 768);        // 192: 2^(5 - e)
    uint64_t* full = reinterpret_cast<uint64_t*>(base + 1536);
    uint64_t* empty = reinterpret_cast<uint64_t*>(base + 1552);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(base + 1568);
    int* s_committed = reinterpret_cast<int*>(base + 1572);
    unsigned char* ops = base + kHeader;

    const GramItem it = items[blockIdx.x];
    const bool diag = it.i0 == it.j0;
    const int h = it.half;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const cx<float>* S = src + it.src;
    // column scales from the largest magnitude of each real column over the row group
    // (k_gram_colmax): rows 0..63 of A the real parts of I, 64..127 the imaginary parts, B
    // the part `half` of J
    // narrow (at most 32 columns, one tile): rows 0..31 of A the real parts, 32..63 the
    // imaginary parts, and B the same 64 rows
    const bool narrow = it.narrow != 0;
    if (tid < 192) {
        int col, part_;
        if (narrow) {
            col = tid < 64 ? (tid & 31) : it.ncols;
            part_ = tid >> 5;
        } else {
            col = tid < 128 ? it.i0 + (tid & 63) : it.j0 + (tid - 128);
            part_ = tid < 64 ? 0 : tid < 128 ? 1 : h;
        }
        colbits[tid] = (col < it.ncols && (tid < 128 || !diag)) ? cmax[it.cmax + 2 * col + part_] : 0u;
    }
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    if (tid == 0) {
        tc::mbar_init(&full[0], 8);
        tc::mbar_init(&full[1], 8);
        tc::mbar_init(&empty[0], 1);
        tc::mbar_init(&empty[1], 1);
        *s_committed = -1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    if (tid < 192) {
        const int E = (int)(colbits[tid] >> 23);   // biased exponent of the maximum (>= 0)
        int e = E - 126;                           // maximum < 2^e
        float sc = 0.0f;
        if (E == 0 || E == 255 || e < -100) e = 0;   // zero, negligible or non-finite (flagged) column
        else sc = __int_as_float((127 + 5 - e) << 23);
        ex[tid] = e;
        scl[tid] = sc;
    }
    __syncthreads();

    const int nsub = (it.r1 - it.r0 + kSub - 1) / kSub;
    bool ok = true;
    if (warp < 8) {
        // producers: thread (p, q) forms rows 8 q .. 8 q + 7 of a step for complex column p
        // of I and (off the diagonal) column p of J's part
        // narrow: threads 0..127, p = column (< 32), q = row group; the others only keep step
        const int p = narrow ? (tid & 31) : (tid & 63), q = narrow ? ((tid >> 5) & 3) : (tid >> 6);
        const bool worker = !narrow || tid < 128;
        const bool colA = worker && it.i0 + p < it.ncols, colB = !narrow && !diag && it.j0 + p < it.ncols;
        const int rim = narrow ? 32 + p : 64 + p;   // A row of the imaginary part
        const float sr = scl[p], si = scl[rim], sb = (diag || narrow) ? 0.0f : scl[128 + p];
        auto load = [&](int step, cx<float> (&za)[8], float (&zb)[8]) {
            const int row0 = it.r0 + step * kSub + 8 * q;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const bool in = row0 + t < it.r1;
                const cx<float>* row = S + (int64_t)(row0 + t) * it.ld;
                za[t] = (colA && in) ? row[it.i0 + p] : cx<float>{0.0f, 0.0f};
                float x = 0.0f;
                if (colB && in) {
                    const cx<float> u = row[it.j0 + p];
                    x = h ? u.y : u.x;
                }
                zb[t] = x;
            }
        };
        cx<float> za[8];
        float zb[8];
        if (nsub > 0) load(0, za, zb);
        for (int sc = 0; sc < nsub; ++sc) {
            const int b = sc & 1;
            cx<float> na[8];
            float nb[8];
            if (sc + 1 < nsub) load(sc + 1, na, nb);   // in flight while this step's digits are formed
            if (sc >= 2 && !tc::mbar_wait(&empty[b], ((sc - 2) >> 1) & 1, kTcWaitPolls)) {
                ok = false;   // the tensor cores never released this buffer
                break;
            }
            unsigned char* Ab = ops + b * (kABytes + kBBytes);
            unsigned char* Bb = Ab + kABytes;
            if (narrow) {
                if (worker) {   // B = A's 64 rows: [Re, Im] of the tile
                    float re[8], im[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        re[t] = za[t].x * sr;
                        im[t] = za[t].y * si;
                    }
                    store_digits(re, Ab, p, Bb, p, q);
                    store_digits(im, Ab, rim, Bb, rim, q);
                }
            } else {
                float re[8], im[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    re[t] = za[t].x * sr;
                    im[t] = za[t].y * si;
                }
                // on the diagonal, J's part is I's own: its digits go to B as well
                store_digits(re, Ab, p, (diag && h == 0) ? Bb : nullptr, p, q);
                store_digits(im, Ab, rim, (diag && h == 1) ? Bb : nullptr, p, q);
            }
            if (!diag && !narrow) {
                float v[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) v[t] = zb[t] * sb;
                store_digits(v, nullptr, 0, Bb, p, q);
            }
            tc::fence_async_smem();   // the generic-proxy stores become visible to the tensor cores
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&full[b]);
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                za[t] = na[t];
                zb[t] = nb[t];
            }
        }
        // every MMA has completed (they complete in order) before the accumulators are read
        if (ok && nsub > 0) ok = tc::mbar_wait(&empty[(nsub - 1) & 1], ((nsub - 1) >> 1) & 1, kTcWaitPolls);
    } else if (lane == 0) {
        // the MMA issuer
        for (int sc = 0; sc < nsub; ++sc) {
            const int b = sc & 1;
            if (!tc::mbar_wait(&full[b], (sc >> 1) & 1, kTcWaitPolls)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            unsigned char* Ab = ops + b * (kABytes + kBBytes);
            const uint32_t a0 = tc::smem_u32(Ab), b0 = tc::smem_u32(Ab + kABytes);
            constexpr uint32_t lboA = (128 / 8) * 128, lboB = (512 / 8) * 128, sbo = 128;
            constexpr uint32_t dA = 128 * kSub * 2;   // bytes per digit of A
#pragma unroll
            for (int ks = 0; ks < kSub / 16; ++ks) {
#pragma unroll 1
                for (int i = 1; i <= kDigits; ++i) {
                    const uint64_t da = tc::sdesc(a0 + (i - 1) * dA + ks * 2 * lboA, lboA, sbo);
                    // the groups g = i + j (TMEM block g - 2) of digits j = 1 .. 9 - i, in runs of
                    // 1, 2 or 4 blocks that start at a multiple of their length (N = 64, 128, 256)
                    for (int blk = i - 1; blk < kDigits;) {
                        int nd = 4;
                        while (nd > 1 && ((blk & (nd - 1)) != 0 || blk + nd > kDigits)) nd >>= 1;
                        const int j1 = blk - i + 2;
                        const uint64_t db = tc::sdesc(b0 + (j1 - 1) * (64 / 8) * 128 + ks * 2 * lboB, lboB, sbo);
                        // digit 1 against digits 1-4 and 5-8 writes all 8 groups: it starts the sums
                        tc::mma_bf16(tmem + (uint32_t)(blk * 64), da, db, tc::idesc_bf16(128, 64 * nd),
                                     sc > 0 || ks > 0 || i > 1);
                        blk += nd;
                    }
                }
            }
            tc::commit(&empty[b]);
            *s_committed = sc;
        }
    }
    ok = __syncthreads_and(ok) != 0;
    tc::fence_after_sync();
    const int committed = *s_committed;

    if (ok && committed >= 0 && narrow) {
        // D (rows m < 64, columns n < 64; real parts first) through shared memory, scaled, then
        // G = Z^* Z: Re G(i, j) = D(i, j) + D(32 + i, 32 + j), Im G(i, j) = D(i, 32 + j) - D(32 + i, j)
        double* Dm = reinterpret_cast<double*>(ops);   // 64 x 64; the operand buffers are free now
        const int qd = warp & 3, ch = warp >> 2;
        if (warp < 8 && qd < 2) {
            const int m = 32 * qd + lane;
            const uint32_t tq = tmem + ((uint32_t)(32 * qd) << 16);
            float hi[32], lo[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.0f;
#pragma unroll 1
            for (int g = 2; g <= kDigits + 1; ++g) {
                float v0[16], v1[16];
                tc::tmem_ld16(tq + (uint32_t)((g - 2) * 64 + 32 * ch), v0);
                tc::tmem_ld16(tq + (uint32_t)((g - 2) * 64 + 32 * ch + 16), v1);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float x = j < 16 ? v0[j] : v1[j - 16];
                    const float s = __fadd_rn(hi[j], x);
                    const float bb = __fsub_rn(s, hi[j]);
                    const float e = __fadd_rn(__fsub_rn(hi[j], __fsub_rn(s, bb)), __fsub_rn(x, bb));
                    hi[j] = s;
                    lo[j] = __fadd_rn(lo[j], e);
                }
            }
            const int em = ex[m];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int e = em + ex[32 * ch + j] - 10;
                Dm[m * 64 + 32 * ch + j] = widen(hi[j], e) + widen(lo[j], e);
            }
        }
        __syncthreads();
        cx<double>* O = part + it.out;   // 32 x 32 tile
        for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
            const int i = idx >> 5, j = idx & 31;
            O[idx] = cx<double>{Dm[i * 64 + j] + Dm[(32 + i) * 64 + 32 + j], Dm[i * 64 + 32 + j] - Dm[(32 + i) * 64 + j]};
        }
    } else if (ok && committed >= 0 && warp < 8) {
        // warp (quarter qd, column half ch): TMEM lane m = row m of D, columns 32 ch .. 32 ch + 31
        const int qd = warp & 3, ch = warp >> 2;
        const int m = 32 * qd + lane;
        const uint32_t tq = tmem + ((uint32_t)(32 * qd) << 16);
        float hi[32], lo[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.0f;
#pragma unroll 1
        for (int g = 2; g <= kDigits + 1; ++g) {
            float v0[16], v1[16];
            tc::tmem_ld16(tq + (uint32_t)((g - 2) * 64 + 32 * ch), v0);
            tc::tmem_ld16(tq + (uint32_t)((g - 2) * 64 + 32 * ch + 16), v1);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float x = j < 16 ? v0[j] : v1[j - 16];
                const float s = __fadd_rn(hi[j], x);                 // two-sum: hi + x = s + e
                const float bb = __fsub_rn(s, hi[j]);
                const float e = __fadd_rn(__fsub_rn(hi[j], __fsub_rn(s, bb)), __fsub_rn(x, bb));
                hi[j] = s;
                lo[j] = __fadd_rn(lo[j], e);
            }
        }
        const int em = ex[m];
        const int i = m & 63;
        const bool top = m < 64;
        const int comp = (h == 0) != top ? 1 : 0;
        const double sgn = (h == 0 && !top) ? -1.0 : 1.0;
        double* o = reinterpret_cast<double*>(part + it.out + (int64_t)i * 64 + 32 * ch) + comp;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            // x_m x_n = 2^(e_m + e_n - 10) y_m y_n
            const int e = em + ex[(diag ? 64 * h : 128) + 32 * ch + j] - 10;
            o[2 * j] = sgn * (widen(hi[j], e) + widen(lo[j], e));
        }
    }
    if (!ok && tid == 0) {
        raise_err(err, ERR_TC_TIMEOUT);
        if (committed >= 0) tc::mbar_wait(&empty[committed & 1], (committed >> 1) & 1, kTcWaitPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// One stack's Gram assembly and pivoted Cholesky (one CTA).
struct CholTask {
    int64_t part;      // cx<double> offset of the stack's first partial tile
    int64_t g;         // cx<double> offset of its c x c working matrix (upper triangle used)
    int64_t dst;       // element offset of the output rows (rout x c, pitch c)
    int32_t ncols, rout, ntile, ngroups;
};

// Pivot threshold relative to the largest diagonal entry of G: the Gram carries absolute
// rounding errors of a few u_64 |Z|^2, so smaller remaining pivots are rounding noise.
constexpr double kCholPivotTol = 16.0 * 2.220446049250313e-16;
constexpr int kCholPanel = 8;   // pivots per panel of the blocked Cholesky

// G (upper triangle) of every stack = the sum of its row groups' partial tiles, in group
// order; grid (element blocks, stacks)
template <int TB>
__global__ void k_gram_sum(const CholTask* __restrict__ tasks, const cx<double>* __restrict__ part,
                           cx<double>* __restrict__ gscr) {
    const CholTask tk = tasks[blockIdx.y];
    const int c = tk.ncols, nt = tk.ntile, ng = tk.ngroups;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)c * c) return;
    const int i = (int)(idx / c), j = (int)(idx - (int64_t)i * c);
    if (i > j) return;
    const int I = i / TB, J = j / TB;
    const int pr = I * nt - (I * (I - 1)) / 2 + (J - I);   // index of tile pair (I, J), I <= J
    const cx<double>* P = part + tk.part + ((int64_t)pr * ng) * TB * TB + (i - I * TB) * TB + (j - J * TB);
    cx<double> v = zero<double>();
    for (int g = 0; g < ng; ++g) v = v + P[(int64_t)g * TB * TB];
    gscr[tk.g + idx] = v;
}

// Pivoted Cholesky of G (upper triangle in gscr, original column order), in panels of
// kCholPanel pivots: within a panel, row j of R is row p_j of G corrected by the panel's
// earlier rows (left-looking) and the remaining diagonal is updated at once; after the panel
// the trailing upper triangle of the remaining columns takes one rank-kCholPanel update
// (right-looking), row by row with consecutive columns per warp.  The panel's rows live in
// shared memory (dynamic: kCholPanel x c complex values).
template <int TB, class TDst>
__global__ void __launch_bounds__(256) k_pchol64(const CholTask* __restrict__ tasks, const cx<double>* __restrict__ part,
                                                 cx<double>* __restrict__ gscr, cx<TDst>* __restrict__ dst,
                                                 unsigned* err) {
    constexpr int CMAX = 512, NB = kCholPanel;
    __shared__ double s_d[CMAX];            // diagonal of the remaining Schur complement
    __shared__ unsigned char s_rem[CMAX];   // 1 while the column is not a pivot
    __shared__ double s_rv[32];
    __shared__ int s_ri[32];
    __shared__ double s_tol;
    extern __shared__ cx<double> s_W[];     // NB x c: the panel's rows of R
    const CholTask tk = tasks[blockIdx.x];
    const int c = tk.ncols;
    cx<double>* G = gscr + tk.g;   // upper triangle summed by k_gram_sum
    cx<TDst>* R = dst + tk.dst;
    for (int l = threadIdx.x; l < c; l += blockDim.x) {
        s_rem[l] = 1;
        s_d[l] = G[(int64_t)l * c + l].x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int l = 0; l < c; ++l) m = fmax(m, s_d[l]);
        s_tol = kCholPivotTol * m;
    }
    __syncthreads();
    const double tol = s_tol;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int j = 0;
    bool done = false;
    while (j < tk.rout && !done) {
        int i = 0;   // rows of this panel
        for (; i < NB && j < tk.rout; ++i, ++j) {
            // pivot: the largest remaining diagonal entry (lowest column on ties)
            double bv = -1.0;
            int bp = c;
            for (int a = threadIdx.x; a < c; a += blockDim.x) {
                if (!s_rem[a]) continue;
                const double v = s_d[a];
                if (!(v == v)) raise_err(err, ERR_TSQR_NONFINITE);
                if (v > bv) {
                    bv = v;
                    bp = a;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int op = __shfl_xor_sync(0xffffffffu, bp, o);
                if (ov > bv || (ov == bv && op < bp)) {
                    bv = ov;
                    bp = op;
                }
            }
            if (lane == 0) {
                s_rv[warp] = bv;
                s_ri[warp] = bp;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double v = s_rv[0];
                int p = s_ri[0];
                for (int q = 1; q < nw; ++q)
                    if (s_rv[q] > v || (s_rv[q] == v && s_ri[q] < p)) {
                        v = s_rv[q];
                        p = s_ri[q];
                    }
                s_rv[0] = v;
                s_ri[0] = p;
                if (v > tol && p < c) s_rem[p] = 0;
            }
            __syncthreads();
            if (!(s_rv[0] > tol)) {   // the rest of G is rounding noise (or the stack is exhausted)
                done = true;
                break;
            }
            const int p = s_ri[0];
            const double rjj = sqrt(s_rv[0]), inv = 1.0 / rjj;
            cx<double>* W = s_W + (int64_t)i * c;
            for (int a = threadIdx.x; a < c; a += blockDim.x) {
                cx<double> v = zero<double>();
                if (a == p) {
                    v = cx<double>{rjj, 0.0};
                } else if (s_rem[a]) {
                    // G'(p, a): this panel's earlier rows are not yet in G
                    v = p <= a ? G[(int64_t)p * c + a] : conj(G[(int64_t)a * c + p]);
                    for (int i2 = 0; i2 < i; ++i2) {
                        const cx<double> wp = s_W[(int64_t)i2 * c + p];
                        fma_cjx(v, cx<double>{-wp.x, -wp.y}, s_W[(int64_t)i2 * c + a]);
                    }
                    v = inv * v;
                    s_d[a] -= v.x * v.x + v.y * v.y;
                }
                W[a] = v;
                R[(int64_t)j * c + a] = cx<TDst>{TDst(v.x), TDst(v.y)};
            }
            __syncthreads();
        }
        if (done || i == 0 || j >= tk.rout) break;
        // trailing update of the remaining columns: G(a, b) -= sum_i conj(W_i(a)) W_i(b), a <= b
        for (int a = warp; a < c; a += nw) {
            if (!s_rem[a]) continue;
            cx<double> wa[NB];
#pragma unroll
            for (int i2 = 0; i2 < NB; ++i2) wa[i2] = i2 < i ? s_W[(int64_t)i2 * c + a] : zero<double>();
            for (int b = a + lane; b < c; b += 32) {
                if (!s_rem[b]) continue;
                cx<double> g = G[(int64_t)a * c + b];
#pragma unroll
                for (int i2 = 0; i2 < NB; ++i2)
                    if (i2 < i) fma_cjx(g, cx<double>{-wa[i2].x, -wa[i2].y}, s_W[(int64_t)i2 * c + b]);
                G[(int64_t)a * c + b] = g;
            }
        }
        __syncthreads();
    }
    // rows past the numerical rank are zero
    for (int idx = j * c + threadIdx.x; idx < tk.rout * c; idx += blockDim.x) R[idx] = zero<TDst>();
}

// G (c x c) from its upper triangle: G(i, j) = conj(G(j, i)) below the diagonal
__global__ void k_gram_full(const cx<double>* __restrict__ up, int c, cx<double>* __restrict__ g) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)c * c) return;
    const int i = (int)(idx / c), j = (int)(idx - (int64_t)i * c);
    g[idx] = i <= j ? up[idx] : conj(up[(int64_t)j * c + i]);
}

template <class TQ, int RPL>
size_t tsqr_smem_bytes(int k) {
    return ((size_t)k * (32 * RPL + 1) + (size_t)kQRNB * k + 2 * kQRNB * kQRNB + kQRNB) * sizeof(cx<TQ>) +
           kQRNB * sizeof(int) + 16;
}

// ----------------------------------------------------------------------------- truncation (FP64)

// ----------------------------------------------------------------------------- leaf orthogonalisation

// Hermitian eigensolver + descending order (NaN-safe): on return lam[i] are the
// eigenvalues of M, order[r] the index of the r-th largest, U the eigenvectors.
//
// FP32 data (X32, Tw given, n >= 8): the sweeps start from an FP32 solution.  The Jacobi first
// runs on an FP32 copy of M (the FP32 pipe is 64x the FP64 one); its eigenvectors U32 are made
// unitary in FP64 by one Newton-Schulz step, U = U32 (I + E), E = (I - U32^* U32) / 2 (E is of
// the order of the FP32 rounding, so it is kept in FP32; U^* U - I drops to ~1e-14), M is
// rotated by U in FP64 (M <- U^* M U, a similarity to FP64 rounding, nearly diagonal) and the
// FP64 sweeps continue from there, with U, to the same stopping rule.  The result is the FP64
// eigendecomposition of M after about two FP64 sweeps instead of six to eight.  (Without the
// Newton-Schulz step the rotation would be a congruence by a matrix unitary only to ~1e-7,
// which moves the small eigenvalues by ~1e-7 |M|.)  X32: n x n complex FP32; Tw: one row of n
// complex FP64 per warp.
template <class T>
__device__ void eig_desc(int n, cx<double>* M, cx<double>* U, JRot<double>* rot, double* red, double* lam,
                         int* order, unsigned* err, cx<float>* X32 = nullptr, cx<double>* Tw = nullptr) {
    bool warm = false;
    if constexpr (std::is_same<T, float>::value) {
        if (X32 != nullptr && Tw != nullptr && n >= 8) {
            const int nn = n * n;
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            cx<float>* M32 = reinterpret_cast<cx<float>*>(U);   // the U area is free until U is formed
            // M scaled by a power of two to magnitudes below 1 (the weighted Grams reach far beyond
            // the FP32 range, and squares of their entries appear in the rotations); the
            // eigenvectors do not change
            double mx = 0.0;
            for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) mx = fmax(mx, fmax(fabs(M[idx].x), fabs(M[idx].y)));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            __syncthreads();
            if (lane == 0) red[warp] = mx;
            __syncthreads();
            mx = 0.0;
            for (int q = 0; q < nw; ++q) mx = fmax(mx, red[q]);
            __syncthreads();
            int ex = 0;
            if (mx > 0.0 && isfinite(mx)) frexp(mx, &ex);
            const double scale = ldexp(1.0, -ex);   // |M| * scale < 1
            for (int idx = threadIdx.x; idx < nn; idx += blockDim.x)
                M32[idx] = cx<float>{float(M[idx].x * scale), float(M[idx].y * scale)};
            __syncthreads();
            herm_jacobi<float>(n, M32, X32, reinterpret_cast<JRot<float>*>(rot), reinterpret_cast<float*>(red), 20,
                               1e-6f);
            __syncthreads();
            for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) U[idx] = cx<double>{double(X32[idx].x), double(X32[idx].y)};
            __syncthreads();
            // E = (I - U^* U) / 2, into the FP32 area
            double emax = 0.0;
            for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
                const int i = idx / n, j = idx - i * n;
                cx<double> g = zero<double>();
                for (int l = 0; l < n; ++l) fma_cjx(g, U[(int64_t)l * n + i], U[(int64_t)l * n + j]);
                const cx<double> ev{0.5 * ((i == j ? 1.0 : 0.0) - g.x), -0.5 * g.y};
                emax = fmax(emax, fmax(fabs(ev.x), fabs(ev.y)));
                if (!(emax <= 1.0)) emax = 2.0;   // NaN
                X32[idx] = cx<float>{float(ev.x), float(ev.y)};
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
            __syncthreads();
            if (lane == 0) red[warp] = emax;
            __syncthreads();
            emax = 0.0;
            for (int q = 0; q < nw; ++q) emax = fmax(emax, red[q]);
            __syncthreads();
            // a start that one Newton-Schulz step cannot make unitary is dropped: the FP64 sweeps
            // then start from the identity (M is untouched so far)
            if (emax <= 1e-4) {
            cx<double>* tmp = Tw + (int64_t)warp * n;
            for (int i = warp; i < n; i += nw) {       // row i of U <- row i of U (I + E)
                for (int j = lane; j < n; j += 32) {
                    cx<double> acc = U[(int64_t)i * n + j];
                    for (int l = 0; l < n; ++l) {
                        const cx<float> e = X32[(int64_t)l * n + j];
                        fma_cx(acc, U[(int64_t)i * n + l], cx<double>{double(e.x), double(e.y)});
                    }
                    tmp[j] = acc;
                }
                __syncwarp();
                for (int j = lane; j < n; j += 32) U[(int64_t)i * n + j] = tmp[j];
                __syncwarp();
            }
            __syncthreads();
            for (int i = warp; i < n; i += nw) {       // row i of M <- row i of M U
                for (int j = lane; j < n; j += 32) {
                    cx<double> acc = zero<double>();
                    for (int l = 0; l < n; ++l) fma_cx(acc, M[(int64_t)i * n + l], U[(int64_t)l * n + j]);
                    tmp[j] = acc;
                }
                __syncwarp();
                for (int j = lane; j < n; j += 32) M[(int64_t)i * n + j] = tmp[j];
                __syncwarp();
            }
            __syncthreads();
            for (int j = warp; j < n; j += nw) {       // column j of M <- column j of U^* M
                for (int i = lane; i < n; i += 32) {
                    cx<double> acc = zero<double>();
                    for (int l = 0; l < n; ++l) fma_cjx(acc, U[(int64_t)l * n + i], M[(int64_t)l * n + j]);
                    tmp[i] = acc;
                }
                __syncwarp();
                for (int i = lane; i < n; i += 32) M[(int64_t)i * n + j] = tmp[i];
                __syncwarp();
            }
            __syncthreads();
            // its Hermitian part (Hermitian up to rounding)
            for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
                const int i = idx / n, j = idx - i * n;
                if (i < j) {
                    const cx<double> a = M[idx], b = M[(int64_t)j * n + i];
                    const cx<double> hh{0.5 * (a.x + b.x), 0.5 * (a.y - b.y)};
                    M[idx] = hh;
                    M[(int64_t)j * n + i] = conj(hh);
                } else if (i == j) {
                    M[idx].y = 0.0;
                }
            }
            __syncthreads();
            warm = true;
            }
        }
    }
    herm_jacobi<double>(n, M, U, rot, red, 40, 1e-15, !warm);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double li = M[(int64_t)i * n + i].x;
        if (!isfinite(li)) {
            raise_err(err, ERR_TRUNC_NONFINITE);
            li = -INFINITY;
        }
        lam[i] = li;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double li = lam[i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += (lam[j] > li || (lam[j] == li && j < i)) ? 1 : 0;
        order[r] = i;
    }
    __syncthreads();
}

// Jacobi workspace of one CTA: shared memory when n <= smem_n, else a global slot
struct EigSpace {
    cx<double>* M;
    cx<double>* U;
    JRot<double>* rot;
    double* lam;
    int* order;
    cx<float>* X32;    // n x n FP32 scratch of the FP32 start (eig_desc)
    cx<double>* Tw;    // kEigWarps rows of n: per-warp staging of the in-place transforms
};

constexpr int kEigWarps = 8;   // warps of the CTAs that call eig_desc (256 threads)

__device__ __forceinline__ EigSpace eig_space(int n, int smem_n, unsigned char* smraw, cx<double>* gslot) {
    EigSpace e;
    if (n <= smem_n) {
        e.M = reinterpret_cast<cx<double>*>(smraw);
        e.U = e.M + (int64_t)smem_n * smem_n;
        e.rot = reinterpret_cast<JRot<double>*>(e.U + (int64_t)smem_n * smem_n);
        e.lam = reinterpret_cast<double*>(e.rot + (smem_n / 2 + 1));
        e.order = reinterpret_cast<int*>(e.lam + smem_n);
        e.X32 = reinterpret_cast<cx<float>*>((reinterpret_cast<uintptr_t>(e.order + smem_n) + 15) &
                                             ~static_cast<uintptr_t>(15));
        e.Tw = reinterpret_cast<cx<double>*>((reinterpret_cast<uintptr_t>(e.X32 + (int64_t)smem_n * smem_n) + 15) &
                                             ~static_cast<uintptr_t>(15));   // 8 smem_n^2 bytes: odd smem_n ends on 8
    } else {
        e.M = gslot;
        e.U = e.M + (int64_t)n * n;
        e.rot = reinterpret_cast<JRot<double>*>(e.U + (int64_t)n * n);
        e.lam = reinterpret_cast<double*>(e.rot + (n / 2 + 1));
        e.order = reinterpret_cast<int*>(e.lam + n);
        e.X32 = reinterpret_cast<cx<float>*>((reinterpret_cast<uintptr_t>(e.order + n) + 15) &
                                             ~static_cast<uintptr_t>(15));
        e.Tw = reinterpret_cast<cx<double>*>((reinterpret_cast<uintptr_t>(e.X32 + (int64_t)n * n) + 15) &
                                             ~static_cast<uintptr_t>(15));   // cx<double> needs 16-byte alignment
    }
    return e;
}

inline size_t eig_smem_bytes(int smem_n) {
    return smem_n > 0 ? 2 * (size_t)smem_n * smem_n * sizeof(cx<double>) + (smem_n / 2 + 1) * sizeof(JRot<double>) +
                            smem_n * (sizeof(double) + sizeof(int)) + 16 + (size_t)smem_n * smem_n * sizeof(cx<float>) +
                            16 + (size_t)kEigWarps * smem_n * sizeof(cx<double>) + 64
                      : 64;
}
inline int64_t eig_global_elems(int n) {   // cx<double> elements of a global Jacobi slot
    int64_t bytes = 2 * (int64_t)n * n * sizeof(cx<double>) + (n / 2 + 1) * sizeof(JRot<double>) +
                    n * (sizeof(double) + sizeof(int)) + 16 + (int64_t)n * n * sizeof(cx<float>) + 16 +
                    (int64_t)kEigWarps * n * sizeof(cx<double>);
    return (bytes + sizeof(cx<double>) - 1) / sizeof(cx<double>) + 4;
}

struct TruncTask {
    int64_t vsrc;      // leaf: V (T) element offset; non-leaf: V-hat scratch (double) offset
    int64_t z;         // Z-hat element offset
    int64_t q;         // output Q / Q-hat (T), row pitch qld
    int64_t c;         // output C (double and T copies), pitch k
    int64_t sig;       // singular values (double)
    int64_t ascratch;  // A = V Z^* scratch (working precision)
    int64_t gslot;     // global Jacobi slot (FP64) when rows exceed the shared-memory size
    int32_t rows, rz, qld, leaf, a, pad;
};

template <class T, bool F64, class FV>
__device__ void truncate_body(const TruncTask& tk, const FV& V, int k, const cx<T>* __restrict__ Z,
                              cx<T>* Ascr, cx<double>* M, cx<double>* U, JRot<double>* rot,
                              double eps, int rule, cx<T>* Q, cx<double>* Cd, cx<T>* Ct,
                              double* sig, int32_t* rank, int* s_order, double* s_lam, unsigned* err,
                              cx<float>* X32, cx<double>* Tw) {
    __shared__ double red[32];
    __shared__ int s_rank;
    const int n = tk.rows, rz = tk.rz;
    const cx<T>* Zt = Z + tk.z;
    // A = V Z^*  (n x rz), working precision
    cta_gemm_fit<T>(n, rz, k, V, [&](int nu, int j) { return conj(Zt[(int64_t)j * k + nu]); },
                [&](int i, int j, cx<T> v) { Ascr[(int64_t)i * rz + j] = v; });
    __syncthreads();
    // left singular vectors of A: FP32 one-sided Jacobi on the rows of A (all-FP32 mixed
    // form), or the FP64 Gram A A^* and a Hermitian Jacobi eigensolver (F64: the FP64 form
    // and the mixed form with FP64 truncation); u(i, r) is entry i of
    // the r-th vector by descending singular value, s_lam[s_order[r]] its squared value
    cx<float>* Jt = reinterpret_cast<cx<float>*>(M);
    if constexpr (std::is_same<T, float>::value && !F64) {
        __shared__ int s_flag;
        rowjac_f32(n, rz, Ascr, rz, Jt, s_lam, s_order, &s_flag, kJacobiSweepsF32, kJacobiTolF32);
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (!isfinite(s_lam[i])) raise_err(err, ERR_TRUNC_NONFINITE);
    } else {
        cta_gemm_fit<double>(n, n, rz, DenseCvt<double, T>{Ascr, rz, false, false},
                             DenseCvt<double, T>{Ascr, rz, true, true},
                             [&](int i, int j, cx<double> v) { M[(int64_t)i * n + j] = v; });
        __syncthreads();
        eig_desc<T>(n, M, U, rot, red, s_lam, s_order, err, X32, Tw);
    }
    auto u = [&](int i, int r) -> cx<T> {
        if constexpr (std::is_same<T, float>::value && !F64) {
            return Jt[(int64_t)s_order[r] * n + i];
        } else {
            const cx<double> v = U[(int64_t)i * n + s_order[r]];
            return cx<T>{T(v.x), T(v.y)};
        }
    };
    const int nsig = min(n, rz);
    if (threadIdx.x == 0) {
        double total = 0;
        for (int r = 0; r < nsig; ++r) total += fmax(s_lam[s_order[r]], 0.0);
        double bound = (rule == DH2_RANK_GLOBAL) ? eps * eps * total : eps * eps;
        int kk = nsig;
        double tail = 0;
        while (kk > 0) {
            double l = fmax(s_lam[s_order[kk - 1]], 0.0);
            if (tail + l <= bound) {
                tail += l;
                --kk;
            } else {
                break;
            }
        }
        if (rule == DH2_RANK_SPECTRAL) {   // smallest k with sigma_{k+1} <= eps
            kk = nsig;
            while (kk > 0 && s_lam[s_order[kk - 1]] <= eps * eps) --kk;
        }
        if (kk > tk.qld) {                 // over the learned cap: the host redoes the pass
            raise_err(err, ERR_RANK_CAP);
            kk = tk.qld;
        }
        s_rank = kk;
        rank[tk.a] = kk;
    }
    for (int r = threadIdx.x; r < nsig; r += blockDim.x) sig[tk.sig + r] = sqrt(fmax(s_lam[s_order[r]], 0.0));
    __syncthreads();
    const int kt = s_rank;
    for (int idx = threadIdx.x; idx < n * kt; idx += blockDim.x) {
        int i = idx / kt, r = idx % kt;
        Q[tk.q + (int64_t)i * tk.qld + r] = u(i, r);
    }
    // C = Q^* V  (kt x k)
    cta_gemm_fit<T>(kt, k, n, [&](int r, int i) { return conj(u(i, r)); }, V,
                [&](int r, int nu, cx<T> v) {
                    Cd[tk.c + (int64_t)r * k + nu] = cx<double>{double(v.x), double(v.y)};
                    Ct[tk.c + (int64_t)r * k + nu] = v;
                });
}

// Truncation of a non-leaf pair: V-hat = [C_t1 E_t1c; C_t2 E_t2c] (working precision),
// A = V-hat Z^*, SVD of A through the FP64 Gram A A^* and a Hermitian Jacobi eigensolver.
template <class T, bool F64>
__global__ void k_truncate(const TruncTask* __restrict__ tasks, int k, const cx<T>* __restrict__ Vhat,
                           const cx<T>* __restrict__ Z, cx<T>* ascr, cx<double>* gscr, int smem_n, double eps,
                           int rule, cx<T>* Q, cx<double>* Cd, cx<T>* Ct, double* sig, int32_t* rank,
                           unsigned* err) {
    extern __shared__ unsigned char smraw[];
    const TruncTask tk = tasks[blockIdx.x];
    const int n = tk.rows;
    EigSpace e = eig_space(n, smem_n, smraw, gscr + tk.gslot);
    truncate_body<T, F64>(tk, Dense<T>{Vhat + tk.vsrc, k, false, false}, k, Z, ascr + tk.ascratch, e.M, e.U, e.rot,
                     eps, rule, Q, Cd, Ct, sig, rank, e.order, e.lam, err, e.X32, e.Tw);
}

struct OrthTask {
    int64_t v, p, r, scr;   // offsets: leaf basis V, output P, output R, global Jacobi slot
    int32_t n, rt;          // rows of V (#t), kept columns of P (min(#t, k))
};

// Leaf basis weights with an explicit orthonormal factor: V V^* = U diag(lam) U^* (FP64
// Gram, Hermitian Jacobi); P = U[:, :rt] (descending eigenvalues), R = P^* V, so V = P R
// and R^* R = V^* V (Eq. basis_weights_def up to a unitary left factor).
template <class T, bool F64>
__global__ void k_leaf_orth(const OrthTask* __restrict__ tasks, int k, cx<T>* V,
                            cx<double>* gscr, int smem_n, cx<T>* P, cx<T>* R, unsigned* err) {
    extern __shared__ unsigned char smraw[];
    __shared__ double red[32];
    const OrthTask tk = tasks[blockIdx.x];
    const int n = tk.n, rt = tk.rt;
    EigSpace e = eig_space(n, smem_n, smraw, gscr + tk.scr);
    cx<T>* Vt = V + tk.v;
    if constexpr (std::is_same<T, float>::value && !F64) {
        // FP32 one-sided Jacobi on the rows of V (rotated in place, V is not used later):
        // V = J W with orthogonal rows w_i, so P = J[:, order], R = W[order, :]
        __shared__ int s_flag;
        cx<float>* Jt = reinterpret_cast<cx<float>*>(e.M);
        rowjac_f32(n, k, Vt, k, Jt, e.lam, e.order, &s_flag, kJacobiSweepsF32, kJacobiTolF32);
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (!isfinite(e.lam[i])) raise_err(err, ERR_TRUNC_NONFINITE);
        for (int idx = threadIdx.x; idx < n * rt; idx += blockDim.x) {
            const int i = idx / rt, j = idx - i * rt;
            P[tk.p + idx] = Jt[(int64_t)e.order[j] * n + i];
        }
        for (int idx = threadIdx.x; idx < rt * k; idx += blockDim.x) {
            const int j = idx / k, nu = idx - j * k;
            R[tk.r + idx] = Vt[(int64_t)e.order[j] * k + nu];
        }
        return;
    }
    cta_gemm_fit<double>(n, n, k, DenseCvt<double, T>{Vt, k, false, false}, DenseCvt<double, T>{Vt, k, true, true},
                     [&](int i, int j, cx<double> v) { e.M[(int64_t)i * n + j] = v; });
    __syncthreads();
    eig_desc<T>(n, e.M, e.U, e.rot, red, e.lam, e.order, err, e.X32, e.Tw);
    for (int idx = threadIdx.x; idx < n * rt; idx += blockDim.x) {
        const int i = idx / rt, j = idx - i * rt;
        const cx<double> u = e.U[(int64_t)i * n + e.order[j]];
        P[tk.p + idx] = cx<T>{T(u.x), T(u.y)};
    }
    cta_gemm_fit<T>(rt, k, n,
                [&](int j, int i) {
                    const cx<double> u = e.U[(int64_t)i * n + e.order[j]];
                    return cx<T>{T(u.x), T(-u.y)};
                },
                Dense<T>{Vt, k, false, false}, [&](int j, int nu, cx<T> v) { R[tk.r + (int64_t)j * k + nu] = v; });
}

struct LeafTruncTask {
    int64_t z, p, r, q, c, sig, scr;   // offsets: Z' (rz x rt), P (n x rt), R (rt x k), Q, C, sigma, slot
    int64_t up;                        // U'[:, :k_tc] (rt x k_tc, pitch qld), kept for the projection
    int32_t rz, rt, n, qld, a, pad;
};

// Truncation of a leaf pair in the coordinates of its orthonormal basis P: with V = P R,
// A = V Z^* has the left singular vectors P U' and the singular values of Z' R-projected,
// where Z'^* Z' = R Z Z^* R^*.  Q = P U'[:, :k_tc], C = Q^* V = U'[:, :k_tc]^* R.
template <class T, bool F64>
__global__ void k_trunc_leaf(const LeafTruncTask* __restrict__ tasks, int k, const cx<T>* __restrict__ Z,
                             const cx<T>* __restrict__ P, const cx<T>* __restrict__ R, cx<double>* gscr,
                             int smem_n, double eps, int rule, cx<T>* Q, cx<double>* Cd, cx<T>* Ct, double* sig,
                             int32_t* rank, cx<T>* Up, unsigned* err) {
    extern __shared__ unsigned char smraw[];
    __shared__ double red[32];
    __shared__ int s_rank;
    const LeafTruncTask tk = tasks[blockIdx.x];
    const int rt = tk.rt, rz = tk.rz, n = tk.n;
    EigSpace e = eig_space(rt, smem_n, smraw, gscr + tk.scr);
    const cx<T>* Zt = Z + tk.z;
    cx<float>* Jt = reinterpret_cast<cx<float>*>(e.M);
    if constexpr (std::is_same<T, float>::value && !F64) {
        // W = Z'^* (rt x rz, rz <= rt) in the U area; FP32 one-sided Jacobi on its rows
        __shared__ int s_flag;
        cx<float>* Wl = reinterpret_cast<cx<float>*>(e.U);
        for (int idx = threadIdx.x; idx < rt * rz; idx += blockDim.x) {
            const int i = idx / rz, j = idx - i * rz;
            Wl[idx] = conj(Zt[(int64_t)j * rt + i]);
        }
        __syncthreads();
        rowjac_f32(rt, rz, Wl, rz, Jt, e.lam, e.order, &s_flag, kJacobiSweepsF32, kJacobiTolF32);
        for (int i = threadIdx.x; i < rt; i += blockDim.x)
            if (!isfinite(e.lam[i])) raise_err(err, ERR_TRUNC_NONFINITE);
    } else {
        // M' = Z'^* Z'  (rt x rt), FP64 Hermitian Jacobi
        cta_gemm_fit<double>(rt, rt, rz,
                             [&](int i, int j) {
                                 cx<T> z = Zt[(int64_t)j * rt + i];
                                 return cx<double>{double(z.x), -double(z.y)};
                             },
                             DenseCvt<double, T>{Zt, rt, false, false},
                             [&](int i, int j, cx<double> v) { e.M[(int64_t)i * rt + j] = v; });
        __syncthreads();
        eig_desc<T>(rt, e.M, e.U, e.rot, red, e.lam, e.order, err, e.X32, e.Tw);
    }
    // entry j of the r-th left singular vector of Z'^* (descending)
    auto u = [&](int j, int r) -> cx<T> {
        if constexpr (std::is_same<T, float>::value && !F64) {
            return Jt[(int64_t)e.order[r] * rt + j];
        } else {
            const cx<double> v = e.U[(int64_t)j * rt + e.order[r]];
            return cx<T>{T(v.x), T(v.y)};
        }
    };
    const int nsig = min(rt, rz);
    if (threadIdx.x == 0) {
        double total = 0;
        for (int r = 0; r < nsig; ++r) total += fmax(e.lam[e.order[r]], 0.0);
        const double bound = (rule == DH2_RANK_GLOBAL) ? eps * eps * total : eps * eps;
        int kk = nsig;
        double tail = 0;
        while (kk > 0) {
            const double l = fmax(e.lam[e.order[kk - 1]], 0.0);
            if (tail + l <= bound) {
                tail += l;
                --kk;
            } else {
                break;
            }
        }
        if (rule == DH2_RANK_SPECTRAL) {   // smallest k with sigma_{k+1} <= eps
            kk = nsig;
            while (kk > 0 && e.lam[e.order[kk - 1]] <= eps * eps) --kk;
        }
        if (kk > tk.qld) {                 // over the learned cap: the host redoes the pass
            raise_err(err, ERR_RANK_CAP);
            kk = tk.qld;
        }
        s_rank = kk;
        rank[tk.a] = kk;
    }
    for (int r = threadIdx.x; r < nsig; r += blockDim.x) sig[tk.sig + r] = sqrt(fmax(e.lam[e.order[r]], 0.0));
    __syncthreads();
    const int kt = s_rank;
    for (int idx = threadIdx.x; idx < rt * kt; idx += blockDim.x) {
        const int j = idx / kt, r = idx - j * kt;
        Up[tk.up + (int64_t)j * tk.qld + r] = u(j, r);
    }
    // Q = P U'[:, :kt]  (n x kt)
    cta_gemm_fit<T>(n, kt, rt, Dense<T>{P + tk.p, rt, false, false}, [&](int j, int r) { return u(j, r); },
                [&](int i, int r, cx<T> v) { Q[tk.q + (int64_t)i * tk.qld + r] = v; });
    // C = U'[:, :kt]^* R  (kt x k)
    cta_gemm_fit<T>(kt, k, rt, [&](int r, int j) { return conj(u(j, r)); },
                Dense<T>{R + tk.r, k, false, false},
                [&](int r, int nu, cx<T> v) {
                    Cd[tk.c + (int64_t)r * k + nu] = cx<double>{double(v.x), double(v.y)};
                    Ct[tk.c + (int64_t)r * k + nu] = v;
                });
}

struct KRowTask {
    int64_t koff, dst;
    int32_t b, rt, rs, pad;
};

// column pass rows of a leaf column cluster: w_b K_b (r_t x r_s), K_b = R_t S_b R_s^*
template <class T>
__global__ void k_stack_from_K(const KRowTask* __restrict__ tasks, int k, const cx<T>* __restrict__ K,
                               const double* __restrict__ bnorm, cx<T>* stack) {
    const KRowTask tk = tasks[blockIdx.x];
    const T w = bnorm[tk.b] > 0.0 ? T(1.0 / bnorm[tk.b]) : T(0);
    for (int idx = threadIdx.x; idx < tk.rt * tk.rs; idx += blockDim.x) {
        const int i = idx / tk.rs, j = idx - i * tk.rs;
        stack[tk.dst + (int64_t)i * k + j] = w * K[tk.koff + idx];
    }
}

struct RhTask {
    int64_t rows_off, r;   // stacked rows (pitch k), R_t
    int32_t rows, rt;
};

// rows <- rows R_t^* in place (first r_t columns): parent rows of a leaf pair projected
// onto its orthonormal basis
template <class T>
__global__ void k_rows_rh(const RhTask* __restrict__ tasks, int k, const cx<T>* __restrict__ R, cx<T>* stack) {
    extern __shared__ unsigned char smraw[];
    cx<T>* row = reinterpret_cast<cx<T>*>(smraw);
    const RhTask tk = tasks[blockIdx.x];
    for (int i = 0; i < tk.rows; ++i) {
        cx<T>* x = stack + tk.rows_off + (int64_t)i * k;
        for (int v = threadIdx.x; v < k; v += blockDim.x) row[v] = x[v];
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int j = warp; j < tk.rt; j += nw) {
            const cx<T>* rj = R + tk.r + (int64_t)j * k;
            cx<T> acc = zero<T>();
            for (int v = lane; v < k; v += 32) fma_cjx(acc, rj[v], row[v]);
            acc = warp_sum(acc);
            if (lane == 0) x[j] = acc;
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------- projection

struct ProjTask {
    int32_t b, kt, ks, leafpair;      // leafpair: both clusters are leaves, S~ = U'_t^* K_b U'_s
    int64_t crow, ccol, dst;
    int64_t koff, upt, ups;           // leaf pairs: K_b and the two U' matrices
    int32_t rt, rs, ldt, lds;
};

template <class T>
__global__ void __launch_bounds__(256, 2) k_project(const ProjTask* __restrict__ tasks, int64_t ntasks,
                          const int32_t* __restrict__ adm_t, const int32_t* __restrict__ adm_s,
                          const int32_t* __restrict__ adm_c, const int32_t* __restrict__ tc_level,
                          const int32_t* __restrict__ dir_off, const double* __restrict__ dirs,
                          const double* __restrict__ nodes, int m, double kappa,
                          const cx<T>* __restrict__ Crow, const cx<T>* __restrict__ Ccol,
                          const cx<T>* __restrict__ Kst, const cx<T>* __restrict__ Upr,
                          const cx<T>* __restrict__ Upc, cx<T>* scratch, cx<T>* Stilde) {
    extern __shared__ unsigned char smraw[];
    const int k = m * m * m;
    cx<T>* T1 = scratch + (int64_t)blockIdx.x * k * k;
    for (int64_t w = blockIdx.x; w < ntasks; w += gridDim.x) {
        const ProjTask tk = tasks[w];
        if (tk.kt == 0 || tk.ks == 0) continue;
        if (tk.leafpair) {
            // S~ = C_t S_b C_s^* with C = U'^* R for leaves: U'_t^* (R_t S_b R_s^*) U'_s
            __syncthreads();
            cta_gemm_fit<T>(tk.kt, tk.rs, tk.rt, [&](int i, int j) { return conj(Upr[tk.upt + (int64_t)j * tk.ldt + i]); },
                        Dense<T>{Kst + tk.koff, tk.rs, false, false},
                        [&](int i, int j, cx<T> v) { T1[(int64_t)i * k + j] = v; });
            __syncthreads();
            cx<T>* out = Stilde + tk.dst;
            const int ks = tk.ks;
            cta_gemm_fit<T>(tk.kt, ks, tk.rs, Dense<T>{T1, k, false, false}, Dense<T>{Upc + tk.ups, tk.lds, false, false},
                        [&](int i, int j, cx<T> v) { out[(int64_t)i * ks + j] = v; });
            __syncthreads();
            continue;
        }
        const int32_t t = adm_t[tk.b], s = adm_s[tk.b], c = adm_c[tk.b];
        const double* cd = dirs + 3 * (dir_off[tc_level[t]] + c);
        __syncthreads();
        const SGen<T> S = load_sgen_tables<T>(t, s, cd, nodes, m, kappa, smraw);
        // T1 = C_t S_b  (kt x k)
        cta_gemm_fit<T>(tk.kt, k, k, Dense<T>{Crow + tk.crow, k, false, false},
                    [&](int mu, int nu) { return S(mu, nu); },
                    [&](int i, int nu, cx<T> v) { T1[(int64_t)i * k + nu] = v; });
        __syncthreads();
        // S~ = T1 C_s^*  (kt x ks)
        cx<T>* out = Stilde + tk.dst;
        const int ks = tk.ks;
        cta_gemm_fit<T>(tk.kt, ks, k, Dense<T>{T1, k, false, false}, Dense<T>{Ccol + tk.ccol, k, true, true},
                    [&](int i, int j, cx<T> v) { out[(int64_t)i * ks + j] = v; });
        __syncthreads();
    }
}

// Projection of a block whose clusters are not both leaves on the tensor cores (k <= 128,
// FP32 data): D1 = (C_t S_b)^T (TMEM columns [0, NT)), then D2 = conj(C_s) D1 (columns
// [NT, 2 NT)), so that S~_b = C_t S_b C_s^* has S~[i][j] = D2[j][i].  One task per CTA.
template <int NT>
__global__ void __launch_bounds__(256, 2) k_project_tc(const ProjTask* __restrict__ tasks,
                                                       const int32_t* __restrict__ adm_t,
                                                       const int32_t* __restrict__ adm_s,
                                                       const int32_t* __restrict__ adm_c,
                                                       const int32_t* __restrict__ tc_level,
                                                       const int32_t* __restrict__ dir_off,
                                                       const double* __restrict__ dirs,
                                                       const double* __restrict__ nodes, int m, double kappa,
                                                       const cx<float>* __restrict__ Crow,
                                                       const cx<float>* __restrict__ Ccol, cx<float>* Stilde,
                                                       unsigned* err) {
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t tc_mbar[1];
    __shared__ uint32_t tc_tmem;
    constexpr int RP = TcTile<NT>::RP;
    const ProjTask tk = tasks[blockIdx.x];
    const int k = m * m * m;
    const int32_t t = adm_t[tk.b], s = adm_s[tk.b], c = adm_c[tk.b];
    const double* cd = dirs + 3 * (dir_off[tc_level[t]] + c);
    float4* Ptab = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
    float4* Qtab = Ptab + 256;
    float* tcbuf = reinterpret_cast<float*>(Qtab + 256);
    load_node_tables(t, s, cd, nodes, m, false, Ptab, Qtab);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3, half = warp >> 2;
    const int kt = tk.kt, ks = tk.ks;
    // k <= 256: nz tiles of 128 rows nu of D1 = (C_t S)^T, ny tiles of 128 rows of S~^T
    const int nz = k > 128 ? 2 : 1, ny = ks > 128 ? 2 : 1;
    const uint32_t ncols = (uint32_t)(2 * nz * NT);
    TcState st;
    tc_begin<NT>(st, tcbuf, tc_mbar, &tc_tmem, ncols);
    for (int z = 0; z < nz; ++z)
        tc_product<NT>(st, (uint32_t)(z * NT), k, GenS<NT>{Ptab + 128 * z, Qtab, k, (float)kappa, k - 128 * z},
                       GenRowsB<NT>{Crow + tk.crow, kt, k, -1.0f});
    for (int y = 0; y < ny; ++y)
        tc_product<NT>(st, (uint32_t)((nz + y) * NT), k, GenRowsA<NT>{Ccol + tk.ccol + (int64_t)128 * y * k, ks - 128 * y, k, k},
                       GenFromTmem<NT>{st.tmem, kt, false});
    if (st.ok) {
        const uint32_t tq = st.tmem + ((uint32_t)(32 * q) << 16);
        cx<float>* out = Stilde + tk.dst;
        for (int y = 0; y < ny; ++y) {
            const int row = 128 * y + 32 * q + lane;
            for (int c0 = half * (RP / 2); c0 < (half + 1) * (RP / 2) && c0 < kt; c0 += 16) {
                float re[16], im[16];
                tc::tmem_ld16(tq + (uint32_t)((nz + y) * NT + c0), re);
                tc::tmem_ld16(tq + (uint32_t)((nz + y) * NT + c0 + RP), im);
                if (row < ks)
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c0 + i < kt) out[(int64_t)(c0 + i) * ks + row] = cx<float>{re[i], im[i]};
            }
        }
    }
    tc_end<NT>(st, err, ncols);
}

// ----------------------------------------------------------------------------- matvec kernels

template <class T, class TX>
__global__ void k_gather(const int32_t* __restrict__ perm, int64_t n, const cx<TX>* __restrict__ x,
                         cx<T>* xt) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    cx<TX> v = x[perm[r]];
    xt[r] = cx<T>{T(v.x), T(v.y)};
}

struct FwdLeaf {
    int64_t q, xh;
    int32_t ld, rows, off, k;
};

// x^_sc = Q_sc^* x|_s for leaf pairs of the column basis
template <class T>
__global__ void k_fwd_leaf(const FwdLeaf* __restrict__ tasks, int64_t ntasks, const cx<T>* __restrict__ Q,
                           const cx<T>* __restrict__ xt, cx<T>* xh) {
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    int64_t w = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5);
    if (w >= ntasks) return;
    const FwdLeaf tk = tasks[w];
    for (int r = 0; r < tk.k; ++r) {
        cx<T> acc = zero<T>();
        for (int i = lane; i < tk.rows; i += 32) fma_cjx(acc, Q[tk.q + (int64_t)i * tk.ld + r], xt[tk.off + i]);
        acc = warp_sum(acc);
        if (lane == 0) xh[tk.xh + r] = acc;
    }
}

struct FwdUp {
    int64_t q, xh, xh0, xh1;
    int32_t ld, k0, k1, k;
};

// x^_sc = F_{s1 c}^* x^_{s1 c'} + F_{s2 c}^* x^_{s2 c'}
template <class T>
__global__ void k_fwd_up(const FwdUp* __restrict__ tasks, int64_t ntasks, const cx<T>* __restrict__ Q,
                         cx<T>* xh) {
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    int64_t w = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5);
    if (w >= ntasks) return;
    const FwdUp tk = tasks[w];
    const int rows = tk.k0 + tk.k1;
    for (int r = 0; r < tk.k; ++r) {
        cx<T> acc = zero<T>();
        for (int i = lane; i < rows; i += 32) {
            cx<T> xv = i < tk.k0 ? xh[tk.xh0 + i] : xh[tk.xh1 + (i - tk.k0)];
            fma_cjx(acc, Q[tk.q + (int64_t)i * tk.ld + r], xv);
        }
        acc = warp_sum(acc);
        if (lane == 0) xh[tk.xh + r] = acc;
    }
}

struct Coup {
    int64_t st, xh;     // S~ offset, x^ offset of the column pair
    int32_t kt, ks;
};

struct Bwd {
    int64_t q, yhp;      // parent Q-hat offset (at this son's first row), parent y^ offset
    int32_t ld, kp;      // parent pitch and rank
};

// y^_{t'c'} += sum over parent directions c+ with sd(c+) = c' of F_{t'c+} y^_{t c+}
template <class T>
__global__ void k_backward(const int32_t* __restrict__ pairs, const int32_t* __restrict__ ptr,
                           const Bwd* __restrict__ items, const int64_t* __restrict__ yh_off,
                           const int32_t* __restrict__ krow, int64_t ntasks, const cx<T>* __restrict__ Q,
                           cx<T>* yh) {
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    int64_t w = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5);
    if (w >= ntasks) return;
    const int32_t a = pairs[w];
    const int k = krow[a];
    for (int i0 = 0; i0 < k; i0 += 32) {
        int i = i0 + lane;
        cx<T> acc = zero<T>();
        if (i < k) {
            for (int e = ptr[w]; e < ptr[w + 1]; ++e) {
                const Bwd it = items[e];
                const cx<T>* row = Q + it.q + (int64_t)i * it.ld;
                for (int r = 0; r < it.kp; ++r) fma_cx(acc, row[r], yh[it.yhp + r]);
            }
            yh[yh_off[a] + i] = yh[yh_off[a] + i] + acc;
        }
    }
}

struct LeafOut {
    int32_t off, rows;
    int32_t qbeg, qend;      // range in the far-field item list
    int32_t sbeg, send;      // range in the nearfield segment list
};
struct LeafQ {
    int64_t q, yh;
    int32_t ld, k;
};
struct LeafSeg {
    int64_t p;               // panel offset of (row 0, first column)
    int32_t ld, xoff, cols, pad;
};

// y[perm[r]] = sum_c Q_tc y^_tc + nearfield rows, one CTA per leaf, one warp per row
template <class T, class TY>
__global__ void k_leaf_out(const LeafOut* __restrict__ leaves, const LeafQ* __restrict__ qitems,
                           const LeafSeg* __restrict__ segs, const cx<T>* __restrict__ Q,
                           const cx<T>* __restrict__ yh, const cx<T>* __restrict__ Pn,
                           const cx<T>* __restrict__ xt, const int32_t* __restrict__ perm, cx<TY>* y) {
    const LeafOut lf = leaves[blockIdx.x];
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x >> 5; i < lf.rows; i += warps) {
        cx<T> acc = zero<T>();
        for (int e = lf.qbeg; e < lf.qend; ++e) {
            const LeafQ it = qitems[e];
            const cx<T>* row = Q + it.q + (int64_t)i * it.ld;
            for (int r = lane; r < it.k; r += 32) fma_cx(acc, row[r], yh[it.yh + r]);
        }
        for (int e = lf.sbeg; e < lf.send; ++e) {
            const LeafSeg sg = segs[e];
            const cx<T>* row = Pn + sg.p + (int64_t)i * sg.ld;
            const cx<T>* xv = xt + sg.xoff;
            for (int j = lane; j < sg.cols; j += 32) fma_cx(acc, row[j], xv[j]);
        }
        acc = warp_sum(acc);
        if (lane == 0) y[perm[lf.off + i]] = cx<TY>{TY(acc.x), TY(acc.y)};
    }
}

// y^_tc = sum_{b in row(t,c)} S~_b x^_sc in two launches.  The couplings of one row pair are
// contiguous (row-list order); the host cuts them into tiles, runs of whole blocks of at
// most kCoupTile bytes (a block larger than that is a tile of its own).  k_coupling_tile:
// one CTA per tile copies it to shared memory with cp.async (many copies in flight per
// thread), forms every (block, row) dot product from shared memory and writes the tile's
// row sums (blocks added in order).  k_coupling_sum: one thread per row of a row pair adds
// its tiles' sums in tile order.  Tiles of similar size balance the load across the SMs;
// every sum has a fixed order (deterministic).
constexpr size_t kCoupTile = 16 * 1024;

struct CoupTile {
    int32_t e0, e1;     // blocks [e0, e1) of the item list
    int32_t kt, pad;    // rows of the row pair
    int64_t out;        // offset of the tile's kt row sums
};

template <class T>
__device__ __forceinline__ void cp_async_elem(cx<T>* dst, const cx<T>* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(cx<T>) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

template <class T, int TILE>
__global__ void __launch_bounds__(256) k_coupling_tile(const CoupTile* __restrict__ tiles,
                                                       const Coup* __restrict__ items, const cx<T>* __restrict__ St,
                                                       const cx<T>* __restrict__ xh, cx<T>* __restrict__ psum) {
    __shared__ __align__(16) cx<T> tile[TILE];
    __shared__ cx<T> part[256];
    const CoupTile tl = tiles[blockIdx.x];
    const int kt = tl.kt, e0 = tl.e0, e1 = tl.e1;
    const Coup first = items[e0], last = items[e1 - 1];
    const int64_t base = first.st, nel = last.st + (int64_t)kt * last.ks - base;
    const bool staged = nel <= TILE;
    if (staged) {
        for (int w = threadIdx.x; w < (int)nel; w += blockDim.x) cp_async_elem<T>(tile + w, St + base + w);
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    cx<T> acc0 = zero<T>(), acc1 = zero<T>();
    const int nw = (e1 - e0) * kt;
    for (int w0 = 0; w0 < nw; w0 += blockDim.x) {
        const int w = w0 + threadIdx.x;
        cx<T> d = zero<T>();
        if (w < nw) {
            const int q = w / kt, i = w - q * kt;
            const Coup it = items[e0 + q];
            const cx<T>* row = staged ? tile + (it.st - base) + (int64_t)i * it.ks : St + it.st + (int64_t)i * it.ks;
            const cx<T>* xv = xh + it.xh;
#pragma unroll 4
            for (int j = 0; j < it.ks; ++j) fma_cx(d, row[j], xv[j]);
        }
        part[threadIdx.x] = d;
        __syncthreads();
        for (int r = threadIdx.x; r < kt; r += blockDim.x) {   // partials (q, r) of this round, in block order
            const int q = (w0 - r + kt - 1) / kt;
            cx<T> sum = zero<T>();
            for (int idx = q * kt + r; idx < w0 + (int)blockDim.x && idx < nw; idx += kt) sum = sum + part[idx - w0];
            if (r < (int)blockDim.x) acc0 = acc0 + sum;
            else acc1 = acc1 + sum;
        }
        __syncthreads();
    }
    if (threadIdx.x < kt) psum[tl.out + threadIdx.x] = acc0;
    if (threadIdx.x + blockDim.x < kt) psum[tl.out + threadIdx.x + blockDim.x] = acc1;
}

// rows of the row pairs with couplings: (row pair offset in y^, first tile sum, tiles, kt)
struct CoupRow {
    int64_t yh, out;
    int32_t ntile, kt;
};

template <class T>
__global__ void k_coupling_sum(const CoupRow* __restrict__ rows, int64_t nrows, int64_t nentries,
                               const int64_t* __restrict__ row_first, const cx<T>* __restrict__ psum, cx<T>* yh) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nentries) return;
    // row pair of entry g: binary search in row_first (first entry index of each row pair)
    int64_t lo = 0, hi = nrows - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (row_first[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const CoupRow r = rows[lo];
    const int i = (int)(g - row_first[lo]);
    cx<T> acc = zero<T>();
    for (int t = 0; t < r.ntile; ++t) acc = acc + psum[r.out + (int64_t)t * r.kt + i];
    yh[r.yh + i] = acc;
}

struct LeafOut2 {
    int64_t poff;            // panel offset (row 0, column 0); even
    int64_t coff;            // offset of the panel's column -> x~ index list
    int32_t off, rows, ld;   // cluster-order row offset, rows, panel width (even)
    int32_t qbeg, qend;      // leaf-basis items
    int32_t nbeg, nend;      // nearfield parts (NearPart) of this leaf
    int32_t pad;
};

// One column chunk of a leaf's nearfield panel: rows x w entries starting at panel offset
// poff (even), row pitch ld; its partial row sums go to pbuf[pofs + i].
struct NearPart {
    int64_t poff, coff, pofs;
    int32_t rows, ld, w, pad;
};
constexpr int kNearChunk = 2048;   // panel columns per part (and x~ values staged per CTA)

// Streams one panel row chunk: sum_j row[j] * xg[j] over this lane's columns (16-byte loads
// for complex FP32).
template <class T>
__device__ __forceinline__ cx<T> near_row_dot(const cx<T>* __restrict__ row, const cx<T>* xg, int w, int lane,
                                              cx<T> a) {
    if constexpr (sizeof(cx<T>) == 8) {
        const float4* r4 = reinterpret_cast<const float4*>(row);
        const int w2 = w >> 1;
#pragma unroll 4
        for (int j = lane; j < w2; j += 32) {
            float4 v = __ldg(r4 + j);
            cx<T> x0 = xg[2 * j], x1 = xg[2 * j + 1];
            fma_cx(a, cx<T>{(T)v.x, (T)v.y}, x0);
            fma_cx(a, cx<T>{(T)v.z, (T)v.w}, x1);
        }
    } else {
#pragma unroll 4
        for (int j = lane; j < w; j += 32) fma_cx(a, row[j], xg[j]);
    }
    return a;
}

// Nearfield partial sums of one panel part (one CTA per part, many per leaf, so that the
// panels of unequal leaves spread over several waves): x~ of the part's columns staged in
// shared memory, each warp streams rows warp, warp + 8, ... and writes pbuf[pofs + i].
template <class T>
__global__ void __launch_bounds__(256) k_near_part(const NearPart* __restrict__ parts,
                                                   const int32_t* __restrict__ colidx,
                                                   const cx<T>* __restrict__ Pn, const cx<T>* __restrict__ xt,
                                                   cx<T>* __restrict__ pbuf) {
    __shared__ cx<T> xg[kNearChunk];
    const NearPart p = parts[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < p.w; j += blockDim.x) xg[j] = xt[colidx[p.coff + j]];
    __syncthreads();
    for (int i = warp; i < p.rows; i += 8) {
        cx<T> a = near_row_dot<T>(Pn + p.poff + (int64_t)i * p.ld, xg, p.w, lane, zero<T>());
        a = warp_sum(a);
        if (lane == 0) pbuf[p.pofs + i] = a;
    }
}

// y[perm[r]] = sum_c Q_tc y^_tc + nearfield row panel: one CTA per leaf.  The x~ values of a
// chunk of panel columns are gathered into shared memory once; each warp then streams its rows
// with 16-byte loads (lane-partial sums kept in registers for up to 8 rows per warp).
// MODE 0: both parts; MODE 1: the nearfield part only (y = panel x~); MODE 2: the leaf-basis
// part plus the nearfield partial sums of the leaf's parts (k_near_part, which runs beside
// the transforms), summed in part order.
template <class T, class TY, int MODE>
__global__ void __launch_bounds__(256) k_leaf_out2(const LeafOut2* __restrict__ leaves,
                                                   const LeafQ* __restrict__ qitems,
                                                   const int32_t* __restrict__ colidx,
                                                   const cx<T>* __restrict__ Q, const cx<T>* __restrict__ yh,
                                                   const cx<T>* __restrict__ Pn, const cx<T>* __restrict__ xt,
                                                   const int32_t* __restrict__ perm, cx<TY>* y,
                                                   const NearPart* __restrict__ parts = nullptr,
                                                   const cx<T>* __restrict__ pbuf = nullptr) {
    constexpr int CH = kNearChunk;
    constexpr int RW = 8;                    // rows per warp per row tile
    __shared__ cx<T> xg[CH];
    const LeafOut2 lf = leaves[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r0 = 0; r0 < lf.rows; r0 += 8 * RW) {
        cx<T> acc[RW];
#pragma unroll
        for (int q = 0; q < RW; ++q) acc[q] = zero<T>();
        for (int c0 = 0; c0 < (MODE == 2 ? 0 : lf.ld); c0 += CH) {
            const int w = min(CH, lf.ld - c0);
            for (int j = threadIdx.x; j < w; j += blockDim.x) xg[j] = xt[colidx[lf.coff + c0 + j]];
            __syncthreads();
#pragma unroll
            for (int q = 0; q < RW; ++q) {
                const int i = r0 + warp + 8 * q;
                if (i >= lf.rows) break;
                acc[q] = near_row_dot<T>(Pn + lf.poff + (int64_t)i * lf.ld + c0, xg, w, lane, acc[q]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < RW; ++q) {
            const int i = r0 + warp + 8 * q;
            if (i >= lf.rows) break;
            cx<T> a = acc[q];
            if (MODE != 1) {
                for (int e = lf.qbeg; e < lf.qend; ++e) {
                    const LeafQ it = qitems[e];
                    const cx<T>* row = Q + it.q + (int64_t)i * it.ld;
                    for (int r = lane; r < it.k; r += 32) fma_cx(a, row[r], yh[it.yh + r]);
                }
            }
            a = warp_sum(a);
            if (lane == 0) {
                if (MODE == 2)
                    for (int e = lf.nbeg; e < lf.nend; ++e) a = a + pbuf[parts[e].pofs + i];
                y[perm[lf.off + i]] = cx<TY>{TY(a.x), TY(a.y)};
            }
        }
    }
}

// ----------------------------------------------------------------------------- complex symmetry

// Copies of per-pair arrays between a pair (t, c) and its mirror (t, -c): the column pass of
// (t, c) is the complex conjugate of the row pass of (t, -c) (G^T = G, D_l = -D_l), and the
// basis weights of (t, -c) are the conjugates of those of (t, c).  One CTA per segment.
struct MirrorSeg {
    int64_t src, dst, n;
};

__global__ void k_mirror_real(const MirrorSeg* __restrict__ segs, const double* __restrict__ src,
                              double* __restrict__ dst) {
    const MirrorSeg m = segs[blockIdx.x];
    for (int64_t i = threadIdx.x; i < m.n; i += blockDim.x) dst[m.dst + i] = src[m.src + i];
}

template <class E, bool CONJ>
__global__ void k_mirror(const MirrorSeg* __restrict__ segs, const E* __restrict__ src, E* __restrict__ dst) {
    const MirrorSeg m = segs[blockIdx.x];
    for (int64_t i = threadIdx.x; i < m.n; i += blockDim.x) {
        E v = src[m.src + i];
        if constexpr (CONJ) v.y = -v.y;
        dst[m.dst + i] = v;
    }
}

// ----------------------------------------------------------------------------- helpers

template <class T>
void upload_vec(DBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
    d.alloc(h.size());
    d.upload(h.data(), h.size(), s);
}

template <class E, bool CONJ>
void mirror_copy(const std::vector<MirrorSeg>& segs, const E* src, E* dst, cudaStream_t s) {
    if (segs.empty()) return;
    DBuf<MirrorSeg> d;
    upload_vec(d, segs, s);
    k_mirror<E, CONJ><<<(unsigned)segs.size(), 128, 0, s>>>(d.p, src, dst);
    DH2_CHECK_LAUNCH("k_mirror");
}

struct StageTimer {
    cudaStream_t s;
    cudaEvent_t ev[2 * ST_COUNT];
    bool used[ST_COUNT] = {false};
    explicit StageTimer(cudaStream_t st) : s(st) {
        for (auto& e : ev) DH2_CHECK_CUDA(cudaEventCreate(&e));
    }
    ~StageTimer() {
        for (auto& e : ev) cudaEventDestroy(e);
    }
    void begin(int i) {
        DH2_CHECK_CUDA(cudaEventRecord(ev[2 * i], s));
        used[i] = true;
    }
    void end(int i) { DH2_CHECK_CUDA(cudaEventRecord(ev[2 * i + 1], s)); }
    void collect(double* out) {
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < ST_COUNT; ++i)
            if (used[i]) {
                float ms = 0;
                DH2_CHECK_CUDA(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
                out[i] += ms;
            }
    }
};

}  // namespace

const char* const kKernelNames[K_COUNT] = {
    "nearfield", "leaf_basis", "transfer", "kron", "stack_blocks", "tsqr", "truncate", "project",
    "mv_gather", "mv_forward", "mv_coupling", "mv_backward", "mv_leaf_out", "tsqr_narrow", "leaf_orth",
    "wqr_chol"};

namespace {
// CUDA-event pairs around individual launches, summed per kernel id on collect().
struct EventLog {
    struct Rec {
        int id;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    void begin(int id, cudaStream_t s) {
        Rec r{id, nullptr, nullptr};
        DH2_CHECK_CUDA(cudaEventCreate(&r.a));
        DH2_CHECK_CUDA(cudaEventCreate(&r.b));
        DH2_CHECK_CUDA(cudaEventRecord(r.a, s));
        recs.push_back(r);
    }
    void end(cudaStream_t s) { DH2_CHECK_CUDA(cudaEventRecord(recs.back().b, s)); }
    void collect(MatrixInfoAcc& info) {
        for (auto& r : recs) {
            DH2_CHECK_CUDA(cudaEventSynchronize(r.b));
            float ms = 0;
            DH2_CHECK_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
            info.kernel_ms[r.id] += ms;
            info.kernel_launches[r.id] += 1;
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        recs.clear();
    }
    ~EventLog() {
        for (auto& r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    }
};
}  // namespace

// ============================================================================= structure download

void download_structure(const Tree& tr, const Structure& st, HostStructure& hs, cudaStream_t s) {
    hs.nc = tr.nc;
    hs.depth = tr.depth;
    hs.offset = tr.offset.to_host(s);
    hs.size = tr.size.to_host(s);
    hs.parent = tr.parent.to_host(s);
    hs.son0 = tr.son0.to_host(s);
    hs.son1 = tr.son1.to_host(s);
    hs.level = tr.level.to_host(s);
    hs.level_start = tr.level_start;
    hs.tc_base = st.tc_base.to_host(s);
    hs.aidx = st.aidx.to_host(s);
    hs.a_t = st.a_t.to_host(s);
    hs.a_c = st.a_c.to_host(s);
    hs.alevel_start = st.alevel_start;
    hs.row_ptr = st.row_ptr.to_host(s);
    hs.row_idx = st.row_idx.to_host(s);
    hs.col_ptr = st.col_ptr.to_host(s);
    hs.col_idx = st.col_idx.to_host(s);
    hs.adm_t = st.adm_t.to_host(s);
    hs.adm_s = st.adm_s.to_host(s);
    hs.adm_c = st.adm_c.to_host(s);
    hs.near_t = st.near_t.to_host(s);
    hs.near_s = st.near_s.to_host(s);
    hs.sd = st.sd.to_host(s);
    hs.dir_off = st.dir_off;
    hs.isd_ptr = st.isd_ptr.to_host(s);
    hs.isd_idx = st.isd_idx.to_host(s);
    hs.nactive = st.nactive;
}

// ============================================================================= Num<T>

// Bytes of K_b stores that builds running now have decided to keep (per process); a build
// holds its share from the decision until its K_b buffer is released.
std::mutex& kb_reserve_mu() {
    static std::mutex mu;
    return mu;
}
int64_t& kb_reserved() {
    static int64_t bytes = 0;
    return bytes;
}
struct KbHold {
    int64_t bytes = 0;
    void acquire(int64_t b) {   // called with kb_reserve_mu() held
        kb_reserved() += b;
        bytes += b;
    }
    void release() {
        if (bytes == 0) return;
        std::lock_guard<std::mutex> lk(kb_reserve_mu());
        kb_reserved() -= bytes;
        bytes = 0;
    }
    ~KbHold() { release(); }
};

template <class T>
class Num : public NumBase {
public:
    Num(const Tree& tr, Structure& st, const HostStructure& hs, const BuildParams& bp)
        : tr_(tr), st_(st), hs_(hs), bp_(bp) {}

    void build(cudaStream_t s) override;
    void matvec(const void* x, void* y, int dtype, cudaStream_t s) override;
    ~Num() override {
        for (auto& g : graph_)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (capture_stream_) cudaStreamDestroy(capture_stream_);
        if (side_stream_) cudaStreamDestroy(side_stream_);
        if (near_stream_) cudaStreamDestroy(near_stream_);
        if (fork_ev_) cudaEventDestroy(fork_ev_);
        if (join_ev_) cudaEventDestroy(join_ev_);
    }
    void matvec_noalloc(const void* x, void* y, int dtype, cudaStream_t s) override;
    void export_pair(int which, int64_t tc, double* out, int64_t cap, int32_t* rows, int32_t* cols,
                     cudaStream_t s) override;
    void export_ranks(int32_t* rr, int32_t* rc, cudaStream_t s) override;
    void set_timing(bool on) override {
        timing_on_ = on;
        for (int i = K_MV_GATHER; i <= K_MV_LEAF_OUT; ++i) {
            info.kernel_ms[i] = 0;
            info.kernel_launches[i] = 0;
        }
    }

private:
    const Tree& tr_;
    Structure& st_;
    const HostStructure& hs_;
    BuildParams bp_;
    int m_ = 0, k_ = 0;
    int64_t n_ = 0, na_ = 0;

    // per active pair (host)
    std::vector<int32_t> lvl_, leaf_, sons_[2], rows_;      // rows_ = #t
    std::vector<int32_t> rR_, rZ_[2], ub_[2], rank_[2];
    std::vector<int64_t> offV_, offE_, offR_, offP_, offK_, offZ_[2], offQ_[2], offC_[2], offSig_[2], ldQ_[2],
        offUp_[2];
    // columns of a pair's total weight: r_t (orthonormal leaf coordinates) or k
    int32_t zcols(int64_t a) const { return leaf_[a] ? rR_[a] : k_; }
    std::vector<std::vector<std::pair<int32_t, int32_t>>> parents_;   // (parent pair, son slot)

    // device data
    DBuf<int32_t> tc_level_;
    DBuf<double> nodes_;
    DBuf<cx<T>> V_, E_, R_, P_, K_, Z_[2], Q_[2], Ct_[2], Up_[2], St_, near_;
    // double layer: leaf column bases W and their weights R_W, P_W (same offsets as V, R, P),
    // element normals (FP64, original order)
    DBuf<cx<T>> W_, RW_, PW_;
    DBuf<double> normals_;
    bool dlp() const { return bp_.layer == DH2_DOUBLE_LAYER; }
    const cx<T>* Rcol() const { return dlp() ? RW_.p : R_.p; }
    const cx<T>* Pcol() const { return dlp() ? PW_.p : P_.p; }
    DBuf<cx<double>> Cd_[2];
    DBuf<double> sig_[2], bnorm_;
    DBuf<int64_t> offR_d_;
    DBuf<int32_t> rR_d_, rank_d_[2];
    DBuf<float> qh_, ql_;
    DBuf<double> x3c_;

    // matvec plan
    DBuf<cx<T>> xt_, xh_, yh_;
    DBuf<FwdLeaf> fwd_leaf_;
    std::vector<std::pair<int64_t, int64_t>> fwd_up_lv_;      // per level range in fwd_up_
    DBuf<FwdUp> fwd_up_;
    DBuf<int32_t> coup_ptr_, krow_d_;
    DBuf<CoupTile> coup_tiles_;         // coupling tiles (k_coupling_tile) and row sums (k_coupling_sum)
    DBuf<CoupRow> coup_rows_;
    DBuf<int64_t> coup_first_;
    DBuf<cx<T>> coup_psum_;
    int64_t n_coup_tiles_ = 0, n_coup_rows_ = 0, n_coup_entries_ = 0;
    void launch_coupling(const cx<T>* xh, cx<T>* yh, cudaStream_t s) {
        if (n_coup_tiles_ == 0) return;
        k_coupling_tile<T, kCoupTile / sizeof(cx<T>)><<<(unsigned)n_coup_tiles_, 256, 0, s>>>(
            coup_tiles_.p, coup_.p, St_.p, xh, coup_psum_.p);
        DH2_CHECK_LAUNCH("k_coupling_tile");
        k_coupling_sum<T><<<grid_for(n_coup_entries_, 256), 256, 0, s>>>(coup_rows_.p, n_coup_rows_, n_coup_entries_,
                                                                        coup_first_.p, coup_psum_.p, yh);
        DH2_CHECK_LAUNCH("k_coupling_sum");
    }
    DBuf<Coup> coup_;
    DBuf<int64_t> yh_off_;
    std::vector<std::pair<int64_t, int64_t>> bwd_lv_;
    DBuf<int32_t> bwd_pairs_, bwd_ptr_;
    DBuf<Bwd> bwd_;
    DBuf<LeafOut> leaf_out_;
    DBuf<LeafQ> leaf_q_;
    DBuf<LeafSeg> leaf_seg_;
    int64_t n_fwd_leaf_ = 0, n_leaves_ = 0;
    std::vector<int64_t> bwd_level_counts_;
    std::vector<int64_t> fwd_up_level_counts_;
    std::vector<std::vector<NearSeg>> leaf_segs_;
    std::vector<int32_t> leaf_order_;
    std::vector<int64_t> leaf_poff_, leaf_coff_;     // per leaf: panel offset, column-list offset
    std::vector<int32_t> leaf_ld_;                   // per leaf: panel width (even)
    std::vector<int64_t> st_off_;                    // per admissible block: S~ offset (row-list order)
    DBuf<int32_t> colidx_;
    DBuf<LeafOut2> leaf_out2_;
    DBuf<NearPart> near_parts_;   // column chunks of the nearfield panels (graph product)
    DBuf<cx<T>> near_pbuf_;       // their partial row sums
    int64_t n_near_parts_ = 0;

    bool timing_on_ = false;
    EventLog ev_;
    DBuf<unsigned> err_;
    void check_err(cudaStream_t s, const char* where) {
        unsigned e = read_scalar(err_.p, s);
        if (e & ERR_TC_TIMEOUT)
            throw Error{DH2_ETIMEOUT, std::string("a bounded tensor-core wait gave up in ") + where + " (code " +
                                          std::to_string(e) + "); the matrix is not usable"};
        if (e) throw Error{DH2_ENUMERIC, std::string("non-finite value in ") + where + " (code " + std::to_string(e) + ")"};
    }
    // test hook (dh2_options.fault): the host sets the device error bit that a device-side
    // timeout or a non-finite value would have set, so that the stage's check reports it
    void inject_fault(cudaStream_t s) {
        unsigned bit = bp_.fault == DH2_FAULT_TIMEOUT ? ERR_TC_TIMEOUT : bp_.fault == DH2_FAULT_NONFINITE ? ERR_TSQR_NONFINITE : 0u;
        if (bit) DH2_CHECK_CUDA(cudaMemcpyAsync(err_.p, &bit, sizeof(bit), cudaMemcpyHostToDevice, s));
    }
    double work_[K_COUNT] = {0};     // algorithmic work accumulated while planning launches
    static constexpr double kEvalFlops = 20.0;   // flop-equivalents per kernel evaluation
    // brackets one launch with CUDA events when `on`
    template <class F>
    void timed(bool on, int id, cudaStream_t s, F&& launch) {
        if (on) ev_.begin(id, s);
        launch();
        if (on) ev_.end(s);
    }

    void layout();
    void layout_trunc(int pass);
    void offsets_trunc(int pass);
    // complex symmetry (dh2_options.symmetry): mirror_[a] is the active pair (t, -c) of the pair
    // a = (t, c); sym_ when the structure is symmetric and the column pass is mirrored.  Of
    // each mirrored couple the pair with the smaller index computes its basis weights.
    std::vector<int32_t> mirror_;
    bool sym_ = false;
    void setup_symmetry(cudaStream_t s);
    bool canonical(int64_t a) const { return !sym_ || mirror_[a] >= a; }
    void mirror_total_weights(cudaStream_t s);
    void mirror_truncation(cudaStream_t s);
    bool capped_[2] = {false, false};
    void analytic(cudaStream_t s);
    void nearfield(cudaStream_t s, EventLog& ev);
    void build_recompression(cudaStream_t s, StageTimer& tm);
    void finish_info();
    void basis_weights(cudaStream_t s);
    void basis_weights_of(bool col, cudaStream_t s);
    void total_weights(int pass, cudaStream_t s);
    template <int NT>
    void launch_stack_blocks(const std::vector<BlockRowTask>& tasks, int pass, cx<T>* stack, cudaStream_t s);
    template <int NT>
    void launch_project_tc(const std::vector<ProjTask>& tasks, cudaStream_t s);
    void launch_matvec(const void* x, void* y, int dtype, cudaStream_t s, bool split = false);
    struct MatvecGraph {
        cudaGraphExec_t exec = nullptr;
        DBuf<unsigned char> x, y;   // the graph's input and output vectors
        int64_t nodes = 0;          // kernels per replay
    };
    MatvecGraph graph_[2];          // complex64, complex128 vectors
    cudaStream_t capture_stream_ = nullptr, side_stream_ = nullptr;
    cudaStream_t near_stream_ = nullptr;   // the nearfield stage, concurrent with the recompression
    bool kstore_ = true;            // K_b kept for the column pass / leaf-pair projection
    KbHold kb_hold_;                // this build's share of the K_b stores of concurrent builds
    cudaEvent_t fork_ev_ = nullptr, join_ev_ = nullptr;
    void truncate(int pass, cudaStream_t s);
    bool truncate_once(int pass, cudaStream_t s);
    void project(cudaStream_t s);
    void project_checked(cudaStream_t s);
    void plan_matvec(cudaStream_t s);
    void tsqr(const std::vector<QRTask>& tasks, const cx<T>* src, cx<T>* dst, cudaStream_t s, const char* where);
    // weight factorisations in FP64 through the Gram matrix and a pivoted Cholesky (the
    // FP64 form and the mixed form with qr_fp64 = 1); qr_fp64 = 2 keeps FP64 Householder
    bool chol_qr() const {
        return std::is_same<T, double>::value ? bp_.qr_fp64 != 2 : bp_.qr_fp64 == 1;
    }
    // Gram tiles of wide FP32 stacks from exact integer digit products on the tensor cores
    bool gram_slices() const { return std::is_same<T, float>::value && chol_qr() && bp_.gram_tc != 0; }
    double gram_mma_flops_[2] = {0.0, 0.0};   // tensor-core work of k_gram_slices: narrow, wide stacks
    // algorithmic flops of one weight factorisation of a stack of `rows` x `cols`
    void qr_work(int64_t rows, int32_t cols) {
        if (rows <= cols) return;   // copied: R = Z
        if (chol_qr()) {   // Hermitian Gram (c(c+1)/2 complex FMA per row) + pivoted Cholesky
            work_[cols <= 32 ? K_TSQR_NARROW : K_TSQR] += 4.0 * rows * cols * (cols + 1.0);
            const double r = (double)std::min<int64_t>(rows, cols);
            work_[K_WQR_CHOL] += 8.0 * (r * cols * cols - r * r * cols + r * r * r / 3.0) / 2.0;
        } else {
            work_[cols <= 32 ? K_TSQR_NARROW : K_TSQR] += 8.0 * rows * cols * cols;
        }
    }
};

// ----------------------------------------------------------------------------- layout

template <class T>
void Num<T>::layout() {
    const auto& h = hs_;
    m_ = bp_.m;
    k_ = m_ * m_ * m_;
    n_ = tr_.n;
    na_ = h.nactive;
    lvl_.resize(na_);
    leaf_.resize(na_);
    rows_.resize(na_);
    sons_[0].assign(na_, -1);
    sons_[1].assign(na_, -1);
    parents_.assign(na_, {});
    for (int64_t a = 0; a < na_; ++a) {
        int32_t t = h.a_t[a], c = h.a_c[a];
        lvl_[a] = h.level[t];
        leaf_[a] = h.son0[t] < 0;
        rows_[a] = h.size[t];
        if (!leaf_[a]) {
            int32_t c1 = h.son_dir(t, c);
            sons_[0][a] = h.pair_of(h.son0[t], c1);
            sons_[1][a] = h.pair_of(h.son1[t], c1);
            if (sons_[0][a] < 0 || sons_[1][a] < 0) throw Error{DH2_ECUDA, "active set not closed"};
            parents_[sons_[0][a]].push_back({(int32_t)a, 0});
            parents_[sons_[1][a]].push_back({(int32_t)a, 1});
        }
    }
    // parent lists in ascending parent direction (sd^{-1} order): parents were visited in
    // active order, which is (t, c) order, so they are already sorted.
    // basis weight rows, bottom-up
    rR_.assign(na_, 0);
    for (int64_t a = na_ - 1; a >= 0; --a) {
        if (leaf_[a])
            rR_[a] = std::min(rows_[a], k_);
        else
            rR_[a] = std::min(rR_[sons_[0][a]] + rR_[sons_[1][a]], k_);
    }
    // total weight rows, top-down
    for (int pass = 0; pass < 2; ++pass) {
        const auto& ptr = pass == 0 ? h.row_ptr : h.col_ptr;
        const auto& idx = pass == 0 ? h.row_idx : h.col_idx;
        rZ_[pass].assign(na_, 0);
        for (int64_t a = 0; a < na_; ++a) {
            int32_t t = h.a_t[a], c = h.a_c[a];
            int32_t tc = h.tc_base[t] + c;
            int64_t rows = 0;
            for (int32_t e = ptr[tc]; e < ptr[tc + 1]; ++e) {
                int32_t b = idx[e];
                int32_t other = pass == 0 ? h.adm_s[b] : h.adm_t[b];
                rows += rR_[h.pair_of(other, c)];
            }
            for (auto& pr : parents_[a]) rows += rZ_[pass][pr.first];
            // leaf pairs keep their total weight in the coordinates of their orthonormal
            // basis (zcols = r_t columns), the others in the interpolation basis (k columns)
            rZ_[pass][a] = (int32_t)std::min<int64_t>(rows, zcols(a));
        }
    }
    // offsets
    auto scan = [&](std::vector<int64_t>& off, auto sizef) {
        off.resize(na_ + 1);
        int64_t acc = 0;
        for (int64_t a = 0; a < na_; ++a) {
            off[a] = acc;
            acc += sizef(a);
        }
        off[na_] = acc;
    };
    scan(offV_, [&](int64_t a) -> int64_t { return leaf_[a] ? (int64_t)rows_[a] * k_ : 0; });
    scan(offE_, [&](int64_t a) -> int64_t { return leaf_[a] ? 0 : 2 * 3 * m_ * m_; });
    scan(offR_, [&](int64_t a) -> int64_t { return (int64_t)rR_[a] * k_; });
    scan(offP_, [&](int64_t a) -> int64_t { return leaf_[a] ? (int64_t)rows_[a] * rR_[a] : 0; });
    {
        const int64_t nb = (int64_t)h.adm_t.size();
        offK_.assign(nb + 1, 0);
        for (int64_t b = 0; b < nb; ++b) {
            const int32_t c = h.adm_c[b];
            offK_[b + 1] = offK_[b] + (int64_t)rR_[h.pair_of(h.adm_t[b], c)] * rR_[h.pair_of(h.adm_s[b], c)];
        }
    }
    for (int pass = 0; pass < 2; ++pass) {
        scan(offZ_[pass], [&](int64_t a) -> int64_t { return (int64_t)rZ_[pass][a] * zcols(a); });
        capped_[pass] = !bp_.rank_cap.empty();
        layout_trunc(pass);
    }
}

// Column bounds of the truncated bases of one pass and the offsets of Q, C, U' and the
// singular values.  The bound ub is min(rows, rank of Z-hat), rows being #t at a leaf and
// the sum of the sons' bounds above; a learned cap, while the pass uses it, lowers it
// further.
template <class T>
void Num<T>::layout_trunc(int pass) {
    if (capped_[pass] && (int64_t)bp_.rank_cap.size() != na_)
        throw Error{DH2_EINVAL, "rank caps: one entry per active pair expected"};
    ub_[pass].assign(na_, 0);
    for (int64_t a = na_ - 1; a >= 0; --a) {
        int32_t rows = leaf_[a] ? rows_[a] : ub_[pass][sons_[0][a]] + ub_[pass][sons_[1][a]];
        ub_[pass][a] = std::min(rows, rZ_[pass][a]);
        if (capped_[pass]) ub_[pass][a] = std::min(ub_[pass][a], std::max(bp_.rank_cap[a], 1));
    }
    offsets_trunc(pass);
}

// Offsets of Q, C, U' and the singular values of one pass from its column bounds ub_.
template <class T>
void Num<T>::offsets_trunc(int pass) {
    auto scan = [&](std::vector<int64_t>& off, auto sizef) {
        off.resize(na_ + 1);
        int64_t acc = 0;
        for (int64_t a = 0; a < na_; ++a) {
            off[a] = acc;
            acc += sizef(a);
        }
        off[na_] = acc;
    };
    ldQ_[pass].resize(na_);
    for (int64_t a = 0; a < na_; ++a) ldQ_[pass][a] = std::max(ub_[pass][a], 1);
    scan(offQ_[pass], [&](int64_t a) -> int64_t {
        int64_t rows = leaf_[a] ? rows_[a] : ub_[pass][sons_[0][a]] + ub_[pass][sons_[1][a]];
        return rows * ldQ_[pass][a];
    });
    scan(offC_[pass], [&](int64_t a) -> int64_t { return (int64_t)ub_[pass][a] * k_; });
    scan(offUp_[pass], [&](int64_t a) -> int64_t { return leaf_[a] ? (int64_t)rR_[a] * ldQ_[pass][a] : 0; });
    scan(offSig_[pass], [&](int64_t a) -> int64_t {
        return leaf_[a] ? rows_[a] : ub_[pass][sons_[0][a]] + ub_[pass][sons_[1][a]];
    });
    rank_[pass].assign(na_, 0);
}

// ----------------------------------------------------------------------------- complex symmetry

// The Galerkin matrix is complex symmetric (g(x, y) = g(y, x) in Eq. 1 and the same basis
// functions on both sides of Eq. 2), the direction sets are point-symmetric (the cube-face
// grid of Remark "construction of directions" is), c_st = -c_ts, and W = V with
// V_{t,-c} = conj(V_{t,c}) (real Lagrange polynomials and weights): then block (s, t, -c) is
// the transpose of block (t, s, c), and the column-pass total weight of (t, c) is the
// conjugate of the row-pass total weight of (t, -c), with everything that the truncation
// derives from it.  The host checks every ingredient on the actual structure (directions up
// to 1e-12, the son maps of the active pairs, the block tree, stack sizes); one failure
// keeps both passes.  (Ties in the nearest-direction rules of the son map and of c_ts go to
// the lowest index, which is not symmetric under c -> -c: directional block trees can fail
// the check.)
template <class T>
void Num<T>::setup_symmetry(cudaStream_t s) {
    sym_ = false;
    mirror_.clear();
    if (!bp_.symmetry || na_ == 0 || dlp()) return;   // the double layer is not symmetric
    const auto& h = hs_;
    const std::vector<double> dirs = st_.dirs.to_host(s);
    const int L = h.depth;
    std::vector<std::vector<int32_t>> mir(L + 1);
    for (int l = 0; l <= L; ++l) {
        const int32_t d0 = h.dir_off[l], nd = h.dir_off[l + 1] - d0;
        mir[l].assign(nd, -1);
        // exact lookup of the negated direction by its coordinates rounded to 2^-30
        std::map<std::array<int64_t, 3>, int32_t> key;
        auto kf = [&](const double* d, double sg) {
            return std::array<int64_t, 3>{std::llround(sg * d[0] * 1073741824.0), std::llround(sg * d[1] * 1073741824.0),
                                          std::llround(sg * d[2] * 1073741824.0)};
        };
        for (int32_t c = 0; c < nd; ++c) key[kf(&dirs[3 * (size_t)(d0 + c)], 1.0)] = c;
        for (int32_t c = 0; c < nd; ++c) {   // -1: no mirror (fails only if an active pair needs it)
            const double* a = &dirs[3 * (size_t)(d0 + c)];
            auto it = key.find(kf(a, -1.0));
            if (it == key.end()) continue;
            const double* b = &dirs[3 * (size_t)(d0 + it->second)];
            if (std::fabs(a[0] + b[0]) <= 1e-12 && std::fabs(a[1] + b[1]) <= 1e-12 && std::fabs(a[2] + b[2]) <= 1e-12)
                mir[l][c] = it->second;
        }
    }
    // active pairs, their sizes, stack heights and sons (the son maps of the active pairs
    // commute with the mirror; ties in the son map elsewhere do not matter)
    std::vector<int32_t> mr(na_);
    for (int64_t a = 0; a < na_; ++a) {
        const int32_t t = h.a_t[a], c = h.a_c[a];
        const int32_t cm = mir[h.level[t]][c];
        if (cm < 0) return;
        const int32_t am = h.pair_of(t, cm);
        if (am < 0) return;
        mr[a] = am;
    }
    for (int64_t a = 0; a < na_; ++a) {
        const int32_t am = mr[a];
        if (mr[am] != a || rR_[am] != rR_[a] || rZ_[1][a] != rZ_[0][am] || rZ_[0][a] != rZ_[1][am]) return;
        if (!leaf_[a] && (sons_[0][am] != mr[sons_[0][a]] || sons_[1][am] != mr[sons_[1][a]])) return;
    }
    // every admissible block (t, s, c) has its transpose (s, t, -c)
    const int64_t nb = (int64_t)h.adm_t.size();
    int64_t dmax = 1;
    for (int l = 0; l <= L; ++l) dmax = std::max<int64_t>(dmax, h.dir_off[l + 1] - h.dir_off[l]);
    const uint64_t ncl = (uint64_t)h.nc;
    auto bkey = [&](int32_t t, int32_t s2, int32_t c) { return ((uint64_t)t * ncl + (uint64_t)s2) * (uint64_t)dmax + c; };
    std::vector<uint64_t> keys(nb);
    for (int64_t b = 0; b < nb; ++b) keys[b] = bkey(h.adm_t[b], h.adm_s[b], h.adm_c[b]);
    std::sort(keys.begin(), keys.end());
    for (int64_t b = 0; b < nb; ++b) {
        const int32_t t = h.adm_t[b], s2 = h.adm_s[b];
        const int32_t cm = mir[h.level[t]][h.adm_c[b]];
        if (cm < 0) return;
        const uint64_t k2 = bkey(s2, t, cm);
        if (!std::binary_search(keys.begin(), keys.end(), k2)) return;
    }
    mirror_.swap(mr);
    sym_ = true;
}

// ----------------------------------------------------------------------------- analytic stage

template <class T>
void Num<T>::analytic(cudaStream_t s) {
    const auto& h = hs_;
    const int32_t nc = tr_.nc;
    nodes_.alloc((size_t)nc * 3 * m_);
    k_cheb_nodes<<<grid_for(nc, kThreads), kThreads, 0, s>>>(tr_.lo.p, tr_.hi.p, nc, m_, nodes_.p);
    DH2_CHECK_LAUNCH("k_cheb_nodes");
    std::vector<int32_t> tcl(hs_.level);
    upload_vec(tc_level_, tcl, s);
    // leaf bases
    std::vector<LeafTask> lt;
    std::vector<TransferTask> tt;
    for (int64_t a = 0; a < na_; ++a) {
        int32_t t = h.a_t[a], c = h.a_c[a];
        int32_t g = h.dir_off[h.level[t]] + c;
        if (leaf_[a]) {
            // direct recompression: the leaf bases are evaluated level by level in basis_weights
            if (!bp_.direct) lt.push_back(LeafTask{t, g, h.offset[t], h.size[t], offV_[a]});
        } else {
            int32_t c1 = h.son_dir(t, c);
            int32_t g1 = h.dir_off[h.level[t] + 1] + c1;
            tt.push_back(TransferTask{t, h.son0[t], g, g1, offE_[a]});
            tt.push_back(TransferTask{t, h.son1[t], g, g1, offE_[a] + 3 * m_ * m_});
        }
    }
    V_.alloc(bp_.direct ? 1 : std::max<int64_t>(offV_[na_], 1));
    E_.alloc(std::max<int64_t>(offE_[na_], 1));
    if (dlp()) {
        normals_.alloc((size_t)3 * std::max<int64_t>(n_, 1));
        k_normals<<<grid_for(n_, kThreads), kThreads, 0, s>>>(tr_.vert.p, tr_.tri.p, n_, normals_.p);
        DH2_CHECK_LAUNCH("k_normals");
        W_.alloc(bp_.direct ? 1 : std::max<int64_t>(offV_[na_], 1));
    }
    if (!lt.empty()) {
        DBuf<LeafTask> d;
        upload_vec(d, lt, s);
        ev_.begin(K_LEAF_BASIS, s);
        k_leaf_basis<T, false><<<(unsigned)lt.size(), 128, 0, s>>>(d.p, tr_.perm.p, tr_.area.p, tr_.x3.p, nodes_.p,
                                                                   st_.dirs.p, m_, bp_.kappa, nullptr, V_.p);
        ev_.end(s);
        DH2_CHECK_LAUNCH("k_leaf_basis");
        if (dlp()) {   // the column bases of the double layer, same layout
            ev_.begin(K_LEAF_BASIS, s);
            k_leaf_basis<T, true><<<(unsigned)lt.size(), 128, 0, s>>>(d.p, tr_.perm.p, tr_.area.p, tr_.x3.p,
                                                                      nodes_.p, st_.dirs.p, m_, bp_.kappa, normals_.p,
                                                                      W_.p);
            ev_.end(s);
            DH2_CHECK_LAUNCH("k_leaf_basis");
        }
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    if (!tt.empty()) {
        DBuf<TransferTask> d;
        upload_vec(d, tt, s);
        ev_.begin(K_TRANSFER, s);
        k_transfer<T><<<(unsigned)tt.size(), 128, 0, s>>>(d.p, nodes_.p, st_.dirs.p, m_, bp_.kappa, E_.p);
        ev_.end(s);
        DH2_CHECK_LAUNCH("k_transfer");
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
    }
}

// ----------------------------------------------------------------------------- nearfield

template <class T>
void Num<T>::nearfield(cudaStream_t s, EventLog& ev) {
    const auto& h = hs_;
    // leaves in offset order: the leaves below a cluster form a contiguous range
    leaf_order_.clear();
    for (int32_t t = 0; t < h.nc; ++t)
        if (h.son0[t] < 0) leaf_order_.push_back(t);
    std::sort(leaf_order_.begin(), leaf_order_.end(),
              [&](int32_t a, int32_t b) { return h.offset[a] < h.offset[b]; });
    std::vector<int32_t> leaf_off(leaf_order_.size());
    for (size_t i = 0; i < leaf_order_.size(); ++i) leaf_off[i] = h.offset[leaf_order_[i]];
    n_leaves_ = (int64_t)leaf_order_.size();
    leaf_segs_.assign(leaf_order_.size(), {});
    for (size_t b = 0; b < h.near_t.size(); ++b) {
        int32_t t = h.near_t[b], s2 = h.near_s[b];
        int32_t lo = h.offset[t], hi = h.offset[t] + h.size[t];
        size_t i0 = std::lower_bound(leaf_off.begin(), leaf_off.end(), lo) - leaf_off.begin();
        for (size_t i = i0; i < leaf_order_.size() && leaf_off[i] < hi; ++i) {
            NearSeg sg{};
            sg.rows = h.size[leaf_order_[i]];
            sg.cols = h.size[s2];
            sg.roff = h.offset[leaf_order_[i]];
            sg.coff = h.offset[s2];
            leaf_segs_[i].push_back(sg);
        }
    }
    // one dense row panel per leaf: its segments side by side, sorted by column offset; the
    // width is padded to even (zero column) so that every row starts on 16 bytes
    std::vector<NearSeg> all;
    int64_t poff = 0, real = 0, ncol = 0;
    leaf_poff_.assign(leaf_order_.size(), 0);
    leaf_coff_.assign(leaf_order_.size(), 0);
    leaf_ld_.assign(leaf_order_.size(), 0);
    for (size_t i = 0; i < leaf_order_.size(); ++i) {
        auto& v = leaf_segs_[i];
        std::sort(v.begin(), v.end(), [](const NearSeg& a, const NearSeg& b) { return a.coff < b.coff; });
        int32_t width = 0;
        for (auto& sg : v) width += sg.cols;
        const int32_t ld = width + (width & 1);
        leaf_poff_[i] = poff;
        leaf_coff_[i] = ncol;
        leaf_ld_[i] = ld;
        int32_t col = 0;
        for (auto& sg : v) {
            sg.ld = ld;
            sg.poff = poff + col;
            sg.cpos = ncol + col;
            col += sg.cols;
            all.push_back(sg);
        }
        ncol += ld;   // a padding column keeps index 0 (its panel entries are zero)
        poff += (int64_t)h.size[leaf_order_[i]] * ld;
        real += (int64_t)h.size[leaf_order_[i]] * width;
    }
    info.near_entries = real;
    near_.alloc(std::max<int64_t>(poff, 1));
    near_.zero(s);
    colidx_.alloc(std::max<int64_t>(ncol, 1));
    colidx_.zero(s);
    {
        // weights of the 7-point rule, to constant memory once per device
        static std::mutex mu;
        static bool ready[64] = {};
        int dev = 0;
        DH2_CHECK_CUDA(cudaGetDevice(&dev));
        DH2_REQUIRE(dev < 64, "nearfield: device ordinal >= 64");
        std::lock_guard<std::mutex> lk(mu);
        if (!ready[dev]) {
            const double s15 = std::sqrt(15.0);
            const double w7[7] = {9.0 / 40.0,           (155.0 - s15) / 1200.0, (155.0 - s15) / 1200.0,
                                  (155.0 - s15) / 1200.0, (155.0 + s15) / 1200.0, (155.0 + s15) / 1200.0,
                                  (155.0 + s15) / 1200.0};
            DH2_CHECK_CUDA(cudaMemcpyToSymbol(c_w7, w7, sizeof(w7)));
            ready[dev] = true;
        }
    }
    QuadRows<T> qr{};
    if constexpr (std::is_same<T, float>::value) {
        qh_.alloc(9 * n_);
        ql_.alloc(9 * n_);
        k_split_quad<<<grid_for(9 * n_, kThreads), kThreads, 0, s>>>(tr_.perm.p, tr_.x3.p, n_, qh_.p, ql_.p);
        DH2_CHECK_LAUNCH("k_split_quad");
        qr.h = qh_.p;
        qr.l = ql_.p;
    } else {
        x3c_.alloc(9 * n_);
        k_cluster_quad<<<grid_for(9 * n_, kThreads), kThreads, 0, s>>>(tr_.perm.p, tr_.x3.p, n_, x3c_.p);
        DH2_CHECK_LAUNCH("k_cluster_quad");
        qr.x = x3c_.p;
    }
    DBuf<NearSeg> dseg;
    upload_vec(dseg, all, s);
    const int64_t chunk = 1 << 22;   // segments (CTAs) per launch
    for (int64_t b0 = 0; b0 < (int64_t)all.size(); b0 += chunk) {
        int64_t cnt = std::min<int64_t>(chunk, (int64_t)all.size() - b0);
        ev.begin(K_NEARFIELD, s);
        if (dlp())
            k_nearfield<T, true><<<(unsigned)cnt, kThreads, 0, s>>>(dseg.p + b0, qr, tr_.perm.p, tr_.area.p, tr_.x3.p,
                                                                    tr_.x7.p, bp_.kappa, normals_.p, near_.p,
                                                                    colidx_.p);
        else
            k_nearfield<T, false><<<(unsigned)cnt, kThreads, 0, s>>>(dseg.p + b0, qr, tr_.perm.p, tr_.area.p,
                                                                     tr_.x3.p, tr_.x7.p, bp_.kappa, nullptr, near_.p,
                                                                     colidx_.p);
        ev.end(s);
        DH2_CHECK_LAUNCH("k_nearfield");
    }
}

// ----------------------------------------------------------------------------- TSQR dispatch

// One launch per column class: stacks of at most 32 or 64 columns run with that pitch,
// so that their shared memory and R scratch are sized for the class instead of for k.
template <int TPC, class TSrc, class TDst>
void launch_tsqr_cols(const std::vector<QRTask>& tasks, int kl, const cx<TSrc>* src, cx<TDst>* dst,
                      DBuf<cx<float>>& scratch, cudaStream_t s, EventLog& ev, unsigned* err, int id) {
    if (tasks.empty()) return;
    const int64_t per = (int64_t)kl * kl;
    const int64_t max_tasks = std::max<int64_t>(1, (int64_t(1) << 31) / (per * (int64_t)sizeof(cx<float>)));
    for (size_t b0 = 0; b0 < tasks.size(); b0 += (size_t)max_tasks) {
        size_t cnt = std::min<size_t>((size_t)max_tasks, tasks.size() - b0);
        std::vector<QRTask> part(tasks.begin() + b0, tasks.begin() + b0 + cnt);
        DBuf<QRTask> d;
        upload_vec(d, part, s);
        scratch.reserve(cnt * per);
        ev.begin(id, s);
        k_tsqr_cols<TPC, 16, TSrc, TDst><<<(unsigned)cnt, 256, 0, s>>>(d.p, kl, src, scratch.p, dst, err);
        ev.end(s);
        DH2_CHECK_LAUNCH("k_tsqr_cols");
    }
}

// The column-parallel kernel with `tpc` threads per column (tpc * kl <= 256).
template <class TSrc, class TDst>
void launch_tsqr_cols_tpc(int tpc, const std::vector<QRTask>& tasks, int kl, const cx<TSrc>* src, cx<TDst>* dst,
                          DBuf<cx<float>>& scratch, cudaStream_t s, EventLog& ev, unsigned* err, int id) {
    switch (tpc) {
        case 1: launch_tsqr_cols<1>(tasks, kl, src, dst, scratch, s, ev, err, id); break;
        case 2: launch_tsqr_cols<2>(tasks, kl, src, dst, scratch, s, ev, err, id); break;
        case 4: launch_tsqr_cols<4>(tasks, kl, src, dst, scratch, s, ev, err, id); break;
        default: launch_tsqr_cols<8>(tasks, kl, src, dst, scratch, s, ev, err, id); break;
    }
}

// Threads per column of each column class: the chosen value if it fits (tpc * class width
// <= 256), else the default (8, 4, 2 for <= 32, <= 64, <= 128 columns).
inline int qr_class_tpc(const int32_t* tpc, int cls) {
    static const int def[3] = {8, 4, 2}, width[3] = {32, 64, 128};
    const int v = tpc ? tpc[cls] : 0;
    return (v == 1 || v == 2 || v == 4 || v == 8) && v * width[cls] <= 256 ? v : def[cls];
}

template <class TSrc, class TQ, class TDst, int RPL>
void launch_tsqr(const std::vector<QRTask>& all_in, int k, const cx<TSrc>* src, cx<TDst>* dst,
                 DBuf<cx<TQ>>& scratch, cudaStream_t s, EventLog& ev, unsigned* err, const int32_t* tpc) {
    const std::vector<QRTask>* pall = &all_in;
    std::vector<QRTask> rest;
    if constexpr (std::is_same<TQ, float>::value) {
        // at most 256 columns: column-parallel kernel (1, 2, 4 or 8 threads per column; the
        // classes of at most 32, 64 and 128 columns take the tuned counts)
        std::vector<QRTask> c1, c2, c4, c8;
        for (const QRTask& t : all_in) {
            if (t.ncols <= 32) c8.push_back(t);
            else if (t.ncols <= 64) c4.push_back(t);
            else if (t.ncols <= 128) c2.push_back(t);
            else if (t.ncols <= 256) c1.push_back(t);
            else rest.push_back(t);
        }
        launch_tsqr_cols_tpc(qr_class_tpc(tpc, 0), c8, 32, src, dst, scratch, s, ev, err, K_TSQR_NARROW);
        launch_tsqr_cols_tpc(qr_class_tpc(tpc, 1), c4, 64, src, dst, scratch, s, ev, err, K_TSQR);
        launch_tsqr_cols_tpc(qr_class_tpc(tpc, 2), c2, 128, src, dst, scratch, s, ev, err, K_TSQR);
        launch_tsqr_cols<1>(c1, 256, src, dst, scratch, s, ev, err, K_TSQR);
        pall = &rest;
    }
    const std::vector<QRTask>& all = *pall;
    std::vector<QRTask> cls[3];
    const int pitch[3] = {std::min(k, 32), std::min(k, 64), k};
    for (const QRTask& t : all) cls[t.ncols <= pitch[0] ? 0 : t.ncols <= pitch[1] ? 1 : 2].push_back(t);
    auto kern = k_tsqr<TSrc, TQ, TDst, RPL>;
    for (int c = 0; c < 3; ++c) {
        const std::vector<QRTask>& tasks = cls[c];
        if (tasks.empty()) continue;
        const int kl = pitch[c];
        const size_t smem = tsqr_smem_bytes<TQ, RPL>(kl);
        ensure_smem(reinterpret_cast<const void*>(kern), smem);
        const int64_t per = (int64_t)kl * kl;
        const int64_t max_tasks = std::max<int64_t>(1, (int64_t(1) << 31) / (per * (int64_t)sizeof(cx<TQ>)));
        for (size_t b0 = 0; b0 < tasks.size(); b0 += (size_t)max_tasks) {
            size_t cnt = std::min<size_t>((size_t)max_tasks, tasks.size() - b0);
            std::vector<QRTask> part(tasks.begin() + b0, tasks.begin() + b0 + cnt);
            DBuf<QRTask> d;
            upload_vec(d, part, s);
            scratch.reserve(cnt * per);
            ev.begin(c == 0 ? K_TSQR_NARROW : K_TSQR, s);
            kern<<<(unsigned)cnt, kThreads, smem, s>>>(d.p, kl, src, scratch.p, dst, err);
            ev.end(s);
            DH2_CHECK_LAUNCH("k_tsqr");
        }
    }
}

// Stacks taller than their group size are split into row groups; the R factors of the
// groups are stacked and factored again (the R factor of a stack is the R factor of the
// stacked R factors of its parts).  Group size: `group` if positive, else 1024 rows;
// never below twice the column count.  (Smaller groups sized to fill every SM, and
// further merge levels for tall merges, both measured slower at 20480 triangles: the
// extra merges cost more than the parallelism they add.)
template <class TS, class TQ, class TD, int RPL>
void tsqr_tree(const std::vector<QRTask>& tasks, int k, int group, const cx<TS>* src, cx<TD>* dst,
               cudaStream_t s, EventLog& ev, unsigned* err, const int32_t* tpc) {
    const int32_t gauto = 1024;
    std::vector<QRTask> direct, groups, merges;
    int64_t mel = 0;   // elements of the merge buffer used so far (group R factors, compact rows)
    for (const QRTask& t : tasks) {
        int32_t g = std::max(group > 0 ? group : gauto, 2 * t.ncols);
        g = (g + 31) / 32 * 32;
        if (t.nrows <= g) {
            direct.push_back(t);
            continue;
        }
        const int64_t m0 = mel;
        int32_t mrows = 0;
        for (int32_t r0 = 0; r0 < t.nrows; r0 += g) {
            // a short last part joins the group before it: every group keeps all its R rows
            // (a group with fewer rows than columns would drop the rows that carry its
            // rounding noise, see k_copy_rows)
            int32_t h = std::min(g, t.nrows - r0);
            if (t.nrows - (r0 + h) > 0 && t.nrows - (r0 + h) < t.ncols) h = t.nrows - r0;
            const int32_t ro = std::min(h, t.ncols);
            groups.push_back(QRTask{t.src + (int64_t)r0 * t.ld, mel, h, ro, t.ncols, t.ld});
            mel += (int64_t)ro * t.ncols;
            mrows += ro;
            if (r0 + h >= t.nrows) break;
        }
        merges.push_back(QRTask{m0, t.dst, mrows, t.rout, t.ncols, t.ncols});
    }
    DBuf<cx<TQ>> scratch, merge;
    launch_tsqr<TS, TQ, TD, RPL>(direct, k, src, dst, scratch, s, ev, err, tpc);
    if (!groups.empty()) {
        merge.alloc((size_t)mel);
        launch_tsqr<TS, TQ, TQ, RPL>(groups, k, src, merge.p, scratch, s, ev, err, tpc);
        launch_tsqr<TQ, TQ, TD, RPL>(merges, k, merge.p, dst, scratch, s, ev, err, tpc);
    }
}

// FP64 Cholesky QR of every stack of a level: stacks of at most 32 columns use 32-column
// Gram tiles (2 x 2 per thread), wider ones 64-column tiles (4 x 4 per thread).  Each
// stack's upper tile pairs are cut into row groups so that the launch has enough CTAs; the
// partial tiles of a stack are summed in group order by the Cholesky kernel (no atomics,
// deterministic).  Stacks are processed in chunks whose scratch stays under 1 GiB.
// Gram matrices (FP64 partial tiles per row group) and pivoted Cholesky factors of the
// stacks.  slices: FP32 stacks take their Gram tiles from k_gram_slices (exact integer
// products on the tensor cores; row groups of at most 2048 rows; two CTAs per tile of a
// stack wider than 32 columns, one for a narrower stack); otherwise k_gram64 forms them
// with FP64 FMAs.  mma_flops[0 | 1] gain the tensor-core work of the narrow | wide stacks.
template <class TS, class TD>
void chol_qr_launch(const std::vector<QRTask>& tasks, const cx<TS>* src, cx<TD>* dst, cudaStream_t s, EventLog& ev,
                    unsigned* err, bool slices = false, double* mma_flops = nullptr,
                    cx<double>* gram_out = nullptr) {
    constexpr int64_t kScratchElems = (int64_t(1) << 30) / (int64_t)sizeof(cx<double>);
    for (int cls = 0; cls < 2; ++cls) {
        const int TB = cls == 0 ? 32 : 64;
        const bool tcg = slices && std::is_same<TS, float>::value;
        const int halves = (tcg && cls == 1) ? 2 : 1;
        std::vector<QRTask> ts;
        for (const QRTask& t : tasks)
            if ((t.ncols <= 32) == (cls == 0) && t.nrows > 0) ts.push_back(t);
        if (ts.empty()) continue;
        double units = 0;
        for (const QRTask& t : ts) {
            const int nt = (t.ncols + TB - 1) / TB;
            units += (double)nt * (nt + 1) / 2 * t.nrows;
        }
        int64_t grows;
        if (tcg) {   // one CTA per SM: about four waves of CTAs, at most 2048 rows each
            grows = std::min<int64_t>(gram_tc::kMaxRows,
                                      std::max<int64_t>(256, (int64_t)std::ceil(units * halves / (152 * 4))));
            grows = (grows + 31) / 32 * 32;
        } else {
            const int64_t want_items = 152 * 12;
            grows = std::max<int64_t>(128, (int64_t)std::ceil(units / want_items));
            grows = (grows + 15) / 16 * 16;
        }
        size_t i0 = 0;
        while (i0 < ts.size()) {
            std::vector<GramItem> items;
            std::vector<CholTask> ct;
            std::vector<ColMaxTask> cmt;   // tcg: column maxima per row group, slices of 256 rows
            int64_t pel = 0, gel = 0, coff = 0;
            size_t i1 = i0;
            for (; i1 < ts.size(); ++i1) {
                const QRTask& t = ts[i1];
                const int nt = (t.ncols + TB - 1) / TB;
                const int ng = (int)((t.nrows + grows - 1) / grows);
                const int64_t tp = (int64_t)nt * (nt + 1) / 2;
                const int64_t need = tp * ng * halves * TB * TB + (int64_t)t.ncols * t.ncols;
                if (i1 > i0 && (pel + gel + need > kScratchElems || ct.size() >= 65535)) break;
                CholTask c{pel, gel, t.dst, t.ncols, t.rout, nt, ng * halves};
                std::vector<int64_t> gcm(ng, 0);
                if (tcg)
                    for (int g = 0; g < ng; ++g) {
                        gcm[g] = coff;
                        coff += 2 * (int64_t)t.ncols;
                        const int32_t r0 = (int32_t)(g * grows);
                        const int32_t r1 = (int32_t)std::min<int64_t>(t.nrows, r0 + grows);
                        for (int32_t rs = r0; rs < r1; rs += 256)
                            cmt.push_back(ColMaxTask{t.src, gcm[g], t.ld, t.ncols, rs, std::min(r1, rs + 256)});
                    }
                for (int I = 0; I < nt; ++I)
                    for (int J = I; J < nt; ++J)
                        for (int g = 0; g < ng; ++g)
                            for (int hf = 0; hf < halves; ++hf) {
                                const int32_t r0 = (int32_t)(g * grows);
                                const int32_t r1 = (int32_t)std::min<int64_t>(t.nrows, r0 + grows);
                                items.push_back(GramItem{t.src, pel, t.ld, t.ncols, r0, r1, I * TB, J * TB, hf,
                                                         cls == 0 ? 1 : 0, gcm[g]});
                                pel += (int64_t)TB * TB;
                                if (tcg && mma_flops) {   // 36 digit products of the real columns
                                    const double mi = 2.0 * std::min(TB, t.ncols - I * TB);
                                    const double nj = (cls == 0 ? 2.0 : 1.0) * std::min(TB, t.ncols - J * TB);
                                    mma_flops[cls] += 2.0 * 36.0 * mi * nj * (r1 - r0);
                                }
                            }
                gel += (int64_t)t.ncols * t.ncols;
                ct.push_back(c);
            }
            for (auto& c : ct) c.g += pel;   // working matrices follow the partial tiles
            DBuf<GramItem> di;
            DBuf<CholTask> dc;
            upload_vec(di, items, s);
            upload_vec(dc, ct, s);
            DBuf<cx<double>> scr((size_t)(pel + gel));
            ev.begin(cls == 0 ? K_TSQR_NARROW : K_TSQR, s);
            if (tcg) {
                if constexpr (std::is_same<TS, float>::value) {
                    DBuf<ColMaxTask> dcm;
                    upload_vec(dcm, cmt, s);
                    DBuf<uint32_t> cmb((size_t)std::max<int64_t>(coff, 1));
                    DH2_CHECK_CUDA(cudaMemsetAsync(cmb.p, 0, (size_t)coff * sizeof(uint32_t), s));
                    k_gram_colmax<<<(unsigned)cmt.size(), 256, 0, s>>>(dcm.p, src, cmb.p, err);
                    DH2_CHECK_LAUNCH("k_gram_colmax");
                    ensure_smem(reinterpret_cast<const void*>(k_gram_slices), gram_tc::kSmemBytes);
                    k_gram_slices<<<(unsigned)items.size(), 288, gram_tc::kSmemBytes, s>>>(di.p, src, cmb.p, scr.p,
                                                                                          err);
                }
            } else if (cls == 0) {
                k_gram64<2, TS><<<(unsigned)items.size(), 256, 0, s>>>(di.p, src, scr.p, err);
            } else {
                k_gram64<4, TS><<<(unsigned)items.size(), 256, 0, s>>>(di.p, src, scr.p, err);
            }
            ev.end(s);
            DH2_CHECK_LAUNCH(tcg ? "k_gram_slices" : "k_gram64");
            ev.begin(K_WQR_CHOL, s);
            int cmax = 1;
            for (const CholTask& c : ct) cmax = std::max(cmax, (int)c.ncols);
            const size_t psm = (size_t)kCholPanel * cmax * sizeof(cx<double>);
            {   // the Gram matrices from the partial tiles, all stacks at once (ct.size() < 65536 per launch)
                const dim3 grid((unsigned)((int64_t(cmax) * cmax + 255) / 256), (unsigned)ct.size());
                if (cls == 0) k_gram_sum<32><<<grid, 256, 0, s>>>(dc.p, scr.p, scr.p);
                else k_gram_sum<64><<<grid, 256, 0, s>>>(dc.p, scr.p, scr.p);
                DH2_CHECK_LAUNCH("k_gram_sum");
            }
            if (cls == 0) {
                ensure_smem(reinterpret_cast<const void*>(k_pchol64<32, TD>), psm);
                k_pchol64<32, TD><<<(unsigned)ct.size(), 256, psm, s>>>(dc.p, scr.p, scr.p, dst, err);
            } else {
                ensure_smem(reinterpret_cast<const void*>(k_pchol64<64, TD>), psm);
                k_pchol64<64, TD><<<(unsigned)ct.size(), 256, psm, s>>>(dc.p, scr.p, scr.p, dst, err);
            }
            ev.end(s);
            DH2_CHECK_LAUNCH("k_pchol64");
            if (gram_out) {   // the summed Gram matrix of the (single) stack, both triangles
                const int c = ct[0].ncols;
                k_gram_full<<<(unsigned)((int64_t(c) * c + 255) / 256), 256, 0, s>>>(scr.p + ct[0].g, c, gram_out);
                DH2_CHECK_LAUNCH("k_gram_full");
            }
            i0 = i1;
        }
    }
}

template <class T>
void Num<T>::tsqr(const std::vector<QRTask>& tasks, const cx<T>* src, cx<T>* dst, cudaStream_t s,
                  const char* where) {
    (void)where;   // the device error word is sticky: the stage that ran this QR reads it once
    // stacks with no more rows than columns are copied (R = Z), the others factored
    std::vector<QRTask> copies, rest;
    for (const QRTask& t : tasks) (t.nrows <= t.ncols ? copies : rest).push_back(t);
    if (!copies.empty()) {
        DBuf<QRTask> d;
        upload_vec(d, copies, s);
        k_copy_rows<T, T><<<(unsigned)copies.size(), 128, 0, s>>>(d.p, src, dst, err_.p);
        DH2_CHECK_LAUNCH("k_copy_rows");
    }
    if (rest.empty()) return;
    if (chol_qr()) {
        chol_qr_launch<T, T>(rest, src, dst, s, ev_, err_.p, gram_slices(), gram_mma_flops_);
        return;
    }
    const bool fp64 = std::is_same<T, double>::value || bp_.qr_fp64;
    if (fp64) {
        if (tsqr_smem_bytes<double, 1>(k_) > 200 * 1024)
            throw Error{DH2_EUNSUPPORTED, "FP64 weight QR supports m <= 6"};
        tsqr_tree<T, double, T, 1>(rest, k_, bp_.qr_group_rows, src, dst, s, ev_, err_.p, bp_.qr_tpc);
    } else if (tsqr_smem_bytes<float, 2>(k_) <= 100 * 1024) {
        tsqr_tree<T, float, T, 2>(rest, k_, bp_.qr_group_rows, src, dst, s, ev_, err_.p, bp_.qr_tpc);
    } else {
        tsqr_tree<T, float, T, 1>(rest, k_, bp_.qr_group_rows, src, dst, s, ev_, err_.p, bp_.qr_tpc);
    }
}

// ----------------------------------------------------------------------------- basis weights

// Basis weights of one basis, bottom-up (Eq. basis_weights_def): col = false the row basis V
// (R_, P_), col = true the column basis W of the double layer (RW_, PW_); the two have the
// same sizes and offsets.
template <class T>
void Num<T>::basis_weights(cudaStream_t s) {
    basis_weights_of(false, s);
    if (dlp()) basis_weights_of(true, s);
    std::vector<int32_t> rr(rR_.begin(), rR_.end());
    upload_vec(rR_d_, rr, s);
    upload_vec(offR_d_, offR_, s);
    check_err(s, "basis weights");
}

template <class T>
void Num<T>::basis_weights_of(bool col, cudaStream_t s) {
    DBuf<cx<T>>& Rb = col ? RW_ : R_;
    DBuf<cx<T>>& Pb = col ? PW_ : P_;
    Rb.alloc(std::max<int64_t>(offR_[na_], 1));
    Pb.alloc(std::max<int64_t>(offP_[na_], 1));
    DBuf<cx<T>> stack;
    DBuf<cx<double>> gscr;
    const int kk = k_;
    for (int l = hs_.depth; l >= 0; --l) {
        std::vector<OrthTask> leafo;
        std::vector<QRTask> innerq;
        std::vector<KronTask> kron;
        int64_t srow = 0, gel = 0;
        int smem_n = 0;
        for (int64_t a = hs_.alevel_start[l]; a < hs_.alevel_start[l + 1]; ++a)
            if (leaf_[a]) smem_n = std::max(smem_n, std::min(rows_[a], 64));
        std::vector<MirrorSeg> mR, mP;   // pairs (t, -c) whose weights are the conjugates of (t, c)'s
        std::vector<LeafTask> vtasks;      // direct recompression: this level's leaf bases
        int64_t vlev = 0;
        for (int64_t a = hs_.alevel_start[l]; a < hs_.alevel_start[l + 1]; ++a) {
            if (!canonical(a)) {
                const int32_t am = mirror_[a];
                mR.push_back(MirrorSeg{offR_[am], offR_[a], (int64_t)rR_[a] * kk});
                if (leaf_[a]) mP.push_back(MirrorSeg{offP_[am], offP_[a], (int64_t)rows_[a] * rR_[a]});
                continue;
            }
            if (leaf_[a]) {
                int64_t voff = offV_[a];
                if (bp_.direct) {
                    const int32_t t = hs_.a_t[a];
                    voff = vlev;
                    vtasks.push_back(LeafTask{t, hs_.dir_off[hs_.level[t]] + hs_.a_c[a], hs_.offset[t], hs_.size[t], voff});
                    vlev += (int64_t)rows_[a] * kk;
                }
                OrthTask o{voff, offP_[a], offR_[a], gel, rows_[a], rR_[a]};
                if (rows_[a] > smem_n) gel += eig_global_elems(rows_[a]);
                leafo.push_back(o);
                work_[K_LEAF_ORTH] += 8.0 * rows_[a] * rows_[a] * kk + 8.0 * rR_[a] * kk * rows_[a];
            } else {
                int32_t s0 = sons_[0][a], s1 = sons_[1][a];
                kron.push_back(KronTask{offR_[s0], offE_[a], srow * kk, rR_[s0], 0});
                kron.push_back(KronTask{offR_[s1], offE_[a] + 3 * m_ * m_, (srow + rR_[s0]) * kk, rR_[s1], 0});
                innerq.push_back(QRTask{srow * kk, offR_[a], rR_[s0] + rR_[s1], rR_[a], kk, kk});
                qr_work(rR_[s0] + rR_[s1], kk);
                work_[K_KRON] += 24.0 * m_ * kk * (rR_[s0] + rR_[s1]);
                srow += rR_[s0] + rR_[s1];
            }
        }
        DBuf<cx<T>> vl;   // direct recompression: evaluated here and orthogonalised at once
        if (!vtasks.empty()) {
            vl.alloc((size_t)vlev);
            DBuf<LeafTask> d;
            upload_vec(d, vtasks, s);
            ev_.begin(K_LEAF_BASIS, s);
            if (col)
                k_leaf_basis<T, true><<<(unsigned)vtasks.size(), 128, 0, s>>>(
                    d.p, tr_.perm.p, tr_.area.p, tr_.x3.p, nodes_.p, st_.dirs.p, m_, bp_.kappa, normals_.p, vl.p);
            else
                k_leaf_basis<T, false><<<(unsigned)vtasks.size(), 128, 0, s>>>(
                    d.p, tr_.perm.p, tr_.area.p, tr_.x3.p, nodes_.p, st_.dirs.p, m_, bp_.kappa, nullptr, vl.p);
            ev_.end(s);
            DH2_CHECK_LAUNCH("k_leaf_basis");
        }
        cx<T>* Vsrc = bp_.direct ? vl.p : (col ? W_.p : V_.p);
        if (!leafo.empty()) {
            gscr.reserve(std::max<int64_t>(gel, 1));
            DBuf<OrthTask> d;
            upload_vec(d, leafo, s);
            const size_t smem = eig_smem_bytes(smem_n);
            // FP64 orthogonalisation with the FP64 weight QRs (and in the FP64 form)
            auto kern = bp_.qr_fp64 ? k_leaf_orth<T, true> : k_leaf_orth<T, false>;
            ensure_smem(reinterpret_cast<const void*>(kern), smem);
            ev_.begin(K_LEAF_ORTH, s);
            kern<<<(unsigned)leafo.size(), kThreads, smem, s>>>(d.p, kk, Vsrc, gscr.p, smem_n, Pb.p, Rb.p, err_.p);
            ev_.end(s);
            DH2_CHECK_LAUNCH("k_leaf_orth");
            check_err(s, "leaf basis weights");
        }
        if (!kron.empty()) {
            stack.reserve(std::max<int64_t>(srow * kk, 1));
            DBuf<KronTask> d;
            upload_vec(d, kron, s);
            size_t smem = (2 * (size_t)kk + 3 * m_ * m_) * sizeof(cx<T>);
            ev_.begin(K_KRON, s);
            k_kron<T, T, T, T><<<(unsigned)kron.size(), kThreads, smem, s>>>(d.p, m_, Rb.p, E_.p, stack.p);
            ev_.end(s);
            DH2_CHECK_LAUNCH("k_kron");
            tsqr(innerq, stack.p, Rb.p, s, "basis weights");
        }
        mirror_copy<cx<T>, true>(mR, Rb.p, Rb.p, s);
        mirror_copy<cx<T>, true>(mP, Pb.p, Pb.p, s);
    }
}

// ----------------------------------------------------------------------------- total weights

template <class T>
template <int NT>
void Num<T>::launch_stack_blocks(const std::vector<BlockRowTask>& tasks, int pass, cx<T>* stack, cudaStream_t s) {
    if (tasks.empty()) return;
    if constexpr (NT > 0 && !std::is_same<T, float>::value) {
        throw Error{DH2_EUNSUPPORTED, "tensor-core coupling products need FP32 data"};
    } else {
        DBuf<BlockRowTask> d;
        upload_vec(d, tasks, s);
        size_t smem = sgen_smem_bytes<T>(m_);
        if constexpr (NT > 0) smem = 128 + 2 * 256 * sizeof(float4) + TcTile<NT>::kOperandBytes;   // 128: alignment
        auto kern = k_stack_blocks<T, NT>;
        ensure_smem(reinterpret_cast<const void*>(kern), smem);
        ev_.begin(K_STACK_BLOCKS, s);
        kern<<<(unsigned)tasks.size(), kThreads, smem, s>>>(d.p, pass == 0, st_.adm_t.p, st_.adm_s.p, st_.adm_c.p,
                                                          tc_level_.p, st_.dir_off_d.p, st_.dirs.p, nodes_.p, m_,
                                                          bp_.kappa, R_.p, Rcol(), offR_d_.p, rR_d_.p, bnorm_.p,
                                                          stack, kstore_ ? K_.p : nullptr, err_.p);
        ev_.end(s);
        DH2_CHECK_LAUNCH("k_stack_blocks");
    }
}

template <class T>
void Num<T>::mirror_total_weights(cudaStream_t s) {
    Z_[1].alloc(std::max<int64_t>(offZ_[1][na_], 1));
    std::vector<MirrorSeg> segs;
    for (int64_t a = 0; a < na_; ++a) {
        const int64_t n = (int64_t)rZ_[1][a] * zcols(a);
        if (n) segs.push_back(MirrorSeg{offZ_[0][mirror_[a]], offZ_[1][a], n});
    }
    mirror_copy<cx<T>, true>(segs, Z_[0].p, Z_[1].p, s);
}

template <class T>
void Num<T>::total_weights(int pass, cudaStream_t s) {
    const auto& h = hs_;
    if (pass == 1 && sym_) {
        mirror_total_weights(s);
        return;
    }
    const auto& ptr = pass == 0 ? h.row_ptr : h.col_ptr;
    const auto& idx = pass == 0 ? h.row_idx : h.col_idx;
    Z_[pass].alloc(std::max<int64_t>(offZ_[pass][na_], 1));
    if (pass == 0) {
        bnorm_.alloc(std::max<int64_t>((int64_t)h.adm_t.size(), 1));
        // K_b = R_t S_b R_s^* is kept for the column pass of leaf columns and the projection of
        // leaf pairs; where the store would not fit (or on request) the tensor-core path
        // recomputes it instead
        kstore_ = true;
        bool can_recompute = false;
        if constexpr (std::is_same<T, float>::value) {
            // the recomputed rows run on the tensor cores only: k <= 128, or k <= 256 with leaf
            // ranks of at most 64 (a TMEM budget of 4 NT columns, NT <= 128)
            int32_t leaf_rank = 0;
            for (int64_t a = 0; a < na_; ++a)
                if (leaf_[a]) leaf_rank = std::max(leaf_rank, rR_[a]);
            can_recompute = bp_.tensor_cores && (k_ <= 128 || (k_ <= 256 && leaf_rank <= 64));
        }
        if (can_recompute && bp_.kb_store != 1) {
            // concurrent builds (the batch) decide one at a time, each against the free memory
            // less what the stores of the others still hold
            std::lock_guard<std::mutex> lk(kb_reserve_mu());
            size_t free_b = 0, total_b = 0;
            DH2_CHECK_CUDA(cudaMemGetInfo(&free_b, &total_b));
            const double bytes = (double)offK_.back() * sizeof(cx<T>);
            const double avail = std::max(0.0, (double)free_b - (double)kb_reserved());
            kstore_ = !(bp_.kb_store == 2 || bytes > 0.25 * avail);
            if (kstore_) kb_hold_.acquire((int64_t)bytes);
        }
        K_.alloc(kstore_ ? std::max<int64_t>(offK_.back(), 1) : 1);
    }
    const int kk = k_;
    const int64_t cap_rows = std::max<int64_t>(
        64, (bp_.workspace_bytes > 0 ? bp_.workspace_bytes : (int64_t(bp_.direct ? 2 : 16) << 30)) /
                ((int64_t)kk * sizeof(cx<T>)));
    DBuf<cx<T>> stack;
    for (int l = 0; l <= h.depth; ++l) {
        int64_t a = h.alevel_start[l];
        const int64_t aend = h.alevel_start[l + 1];
        while (a < aend) {
            std::vector<BlockRowTask> btasks;   // rows generated from S_b
            std::vector<KRowTask> ktasks;       // column pass, leaf column cluster: rows from K_b
            std::vector<KronTask> ptasks;       // rows inherited from the father
            std::vector<RhTask> rhtasks;        // father rows of leaf pairs, projected
            std::vector<QRTask> qtasks;
            int64_t srow = 0;
            for (; a < aend; ++a) {
                const int32_t t = h.a_t[a], c = h.a_c[a], tc = h.tc_base[t] + c;
                int64_t rows = 0;
                for (int32_t e = ptr[tc]; e < ptr[tc + 1]; ++e) {
                    int32_t other = pass == 0 ? h.adm_s[idx[e]] : h.adm_t[idx[e]];
                    rows += rR_[h.pair_of(other, c)];
                }
                for (auto& pr : parents_[a]) rows += rZ_[pass][pr.first];
                if (srow > 0 && srow + rows > cap_rows) break;   // next group
                const int64_t r0 = srow;
                const int32_t zc = zcols(a);
                for (int32_t e = ptr[tc]; e < ptr[tc + 1]; ++e) {
                    const int32_t b = idx[e];
                    const int32_t other = pass == 0 ? h.adm_s[b] : h.adm_t[b];
                    const int32_t ao = h.pair_of(other, c);
                    if (pass == 1 && leaf_[a] && kstore_) {
                        // rows w K_b (r_t x r_s) from the row pass, no coupling evaluation
                        ktasks.push_back(KRowTask{offK_[b], srow * kk, b, rR_[ao], rR_[a], 0});
                    } else if (pass == 1 && leaf_[a]) {
                        // the same rows, K_b recomputed on the tensor cores (other = s, own = t)
                        btasks.push_back(BlockRowTask{b, (int32_t)a, ao, 2, srow * kk, 0});
                        work_[K_STACK_BLOCKS] += kEvalFlops * kk * kk + 8.0 * rR_[a] * kk * kk +
                                                 8.0 * rR_[ao] * kk * rR_[a];
                    } else {
                        btasks.push_back(BlockRowTask{b, ao, (int32_t)a, pass == 0 ? (int32_t)leaf_[a] : 0,
                                                      srow * kk, pass == 0 ? offK_[b] : 0});
                        work_[K_STACK_BLOCKS] += kEvalFlops * kk * kk + 8.0 * rR_[ao] * kk * kk +
                                                 (pass == 0 ? 8.0 * rR_[a] * kk * rR_[ao] : 0.0);
                    }
                    srow += rR_[ao];
                }
                for (auto& pr : parents_[a]) {
                    const int32_t ap = pr.first;
                    if (rZ_[pass][ap] == 0) continue;
                    ptasks.push_back(KronTask{offZ_[pass][ap], offE_[ap] + (int64_t)pr.second * 3 * m_ * m_,
                                              srow * kk, rZ_[pass][ap], 1});
                    if (leaf_[a]) rhtasks.push_back(RhTask{srow * kk, offR_[a], rZ_[pass][ap], rR_[a]});
                    work_[K_KRON] += 24.0 * m_ * kk * rZ_[pass][ap];
                    srow += rZ_[pass][ap];
                }
                qtasks.push_back(QRTask{r0 * kk, offZ_[pass][a], (int32_t)(srow - r0), rZ_[pass][a], zc, kk});
                qr_work(srow - r0, zc);
            }
            stack.reserve(std::max<int64_t>(srow * kk, 1));
            if (!btasks.empty()) {
                bool tcore = false;
                if constexpr (std::is_same<T, float>::value) tcore = bp_.tensor_cores && kk <= 256;
                if (tcore) {
                    // tensor-core tiles by the rank of the R factor: N = 2 x (32 | 64 | 128); with
                    // k > 128 (two M tiles, 4 NT TMEM columns) ranks above 64 stay on the CUDA cores
                    std::vector<BlockRowTask> cls[3], simt;
                    for (const BlockRowTask& b : btasks) {
                        const int32_t ro = rR_[b.other];
                        const int c = ro <= 32 ? 0 : ro <= 64 ? 1 : 2;
                        if (c == 2 && kk > 128) simt.push_back(b);
                        else cls[c].push_back(b);
                    }
                    launch_stack_blocks<64>(cls[0], pass, stack.p, s);
                    launch_stack_blocks<128>(cls[1], pass, stack.p, s);
                    launch_stack_blocks<256>(cls[2], pass, stack.p, s);
                    launch_stack_blocks<0>(simt, pass, stack.p, s);
                } else {
                    launch_stack_blocks<0>(btasks, pass, stack.p, s);
                }
            }
            if (!ktasks.empty()) {
                DBuf<KRowTask> d;
                upload_vec(d, ktasks, s);
                k_stack_from_K<T><<<(unsigned)ktasks.size(), 128, 0, s>>>(d.p, kk, K_.p, bnorm_.p, stack.p);
                DH2_CHECK_LAUNCH("k_stack_from_K");
            }
            if (!ptasks.empty()) {
                DBuf<KronTask> d;
                upload_vec(d, ptasks, s);
                size_t smem = (2 * (size_t)kk + 3 * m_ * m_) * sizeof(cx<T>);
                ev_.begin(K_KRON, s);
                k_kron<T, T, T, T><<<(unsigned)ptasks.size(), kThreads, smem, s>>>(d.p, m_, Z_[pass].p, E_.p,
                                                                                   stack.p);
                ev_.end(s);
                DH2_CHECK_LAUNCH("k_kron");
            }
            if (!rhtasks.empty()) {
                DBuf<RhTask> d;
                upload_vec(d, rhtasks, s);
                // the leaf's own basis: V in the rows pass, W in the columns pass
                k_rows_rh<T><<<(unsigned)rhtasks.size(), kThreads, (size_t)kk * sizeof(cx<T>), s>>>(
                    d.p, kk, pass == 0 ? R_.p : Rcol(), stack.p);
                DH2_CHECK_LAUNCH("k_rows_rh");
            }
            tsqr(qtasks, stack.p, Z_[pass].p, s, pass == 0 ? "total weights (rows)" : "total weights (columns)");
        }
    }
    check_err(s, pass == 0 ? "total weights (rows)" : "total weights (columns)");
}

// ----------------------------------------------------------------------------- truncation

// The column pass as the conjugate of the row pass at the mirrored pairs: bounds, ranks,
// Q / F, C, U' and singular values.
template <class T>
void Num<T>::mirror_truncation(cudaStream_t s) {
    for (int64_t a = 0; a < na_; ++a) ub_[1][a] = ub_[0][mirror_[a]];
    offsets_trunc(1);
    Q_[1].alloc(std::max<int64_t>(offQ_[1][na_], 1));
    Up_[1].alloc(std::max<int64_t>(offUp_[1][na_], 1));
    Cd_[1].alloc(std::max<int64_t>(offC_[1][na_], 1));
    if constexpr (std::is_same<T, float>::value) Ct_[1].alloc(std::max<int64_t>(offC_[1][na_], 1));
    sig_[1].alloc(std::max<int64_t>(offSig_[1][na_], 1));
    std::vector<MirrorSeg> q, c, u, g;
    for (int64_t a = 0; a < na_; ++a) {
        const int32_t am = mirror_[a];
        rank_[1][a] = rank_[0][am];
        auto seg = [&](std::vector<MirrorSeg>& v, const std::vector<int64_t>* off) {
            const int64_t n = off[0][am + 1] - off[0][am];
            if (n != off[1][a + 1] - off[1][a]) throw Error{DH2_ECUDA, "mirrored truncation: sizes differ"};
            if (n) v.push_back(MirrorSeg{off[0][am], off[1][a], n});
        };
        seg(q, offQ_);
        seg(c, offC_);
        seg(u, offUp_);
        seg(g, offSig_);
    }
    mirror_copy<cx<T>, true>(q, Q_[0].p, Q_[1].p, s);
    mirror_copy<cx<T>, true>(u, Up_[0].p, Up_[1].p, s);
    mirror_copy<cx<double>, true>(c, Cd_[0].p, Cd_[1].p, s);
    if constexpr (std::is_same<T, float>::value) mirror_copy<cx<float>, true>(c, Ct_[0].p, Ct_[1].p, s);
    {
        if (!g.empty()) {   // singular values (real)
            DBuf<MirrorSeg> d;
            upload_vec(d, g, s);
            k_mirror_real<<<(unsigned)g.size(), 128, 0, s>>>(d.p, sig_[0].p, sig_[1].p);
            DH2_CHECK_LAUNCH("k_mirror");
        }
    }
    upload_vec(rank_d_[1], rank_[1], s);
}

template <class T>
void Num<T>::truncate(int pass, cudaStream_t s) {
    if (pass == 1 && sym_) {
        mirror_truncation(s);
        const int64_t cb = std::is_same<T, float>::value ? (int64_t)sizeof(cx<float>) : 0;
        info.truncation_bytes += offQ_[1][na_] * (int64_t)sizeof(cx<T>) + offUp_[1][na_] * (int64_t)sizeof(cx<T>) +
                                 offC_[1][na_] * ((int64_t)sizeof(cx<double>) + cb) + offSig_[1][na_] * 8;
        return;
    }
    while (!truncate_once(pass, s)) {
        // a rank exceeded its learned cap: redo the pass with the structural bounds
        err_.zero(s);
        capped_[pass] = false;
        layout_trunc(pass);
        ++info.rank_cap_retries;
    }
    const int64_t cb = std::is_same<T, float>::value ? (int64_t)sizeof(cx<float>) : 0;
    info.truncation_bytes += offQ_[pass][na_] * (int64_t)sizeof(cx<T>) + offUp_[pass][na_] * (int64_t)sizeof(cx<T>) +
                             offC_[pass][na_] * ((int64_t)sizeof(cx<double>) + cb) + offSig_[pass][na_] * 8;
}

// One truncation pass, level by level bottom-up; false when a rank exceeded its cap.
template <class T>
bool Num<T>::truncate_once(int pass, cudaStream_t s) {
    const auto& h = hs_;
    const int kk = k_;
    Q_[pass].alloc(std::max<int64_t>(offQ_[pass][na_], 1));
    Up_[pass].alloc(std::max<int64_t>(offUp_[pass][na_], 1));
    Cd_[pass].alloc(std::max<int64_t>(offC_[pass][na_], 1));
    if constexpr (std::is_same<T, float>::value) Ct_[pass].alloc(std::max<int64_t>(offC_[pass][na_], 1));
    sig_[pass].alloc(std::max<int64_t>(offSig_[pass][na_], 1));
    rank_d_[pass].alloc(std::max<int64_t>(na_, 1));
    cx<T>* Ct = nullptr;
    if constexpr (std::is_same<T, float>::value) Ct = Ct_[pass].p;
    else Ct = reinterpret_cast<cx<T>*>(Cd_[pass].p);
    DBuf<cx<T>> vhat, ascr;
    DBuf<cx<double>> gscr, lscr;
    for (int l = h.depth; l >= 0; --l) {
        const int64_t a0 = h.alevel_start[l], a1 = h.alevel_start[l + 1];
        if (a1 == a0) continue;
        std::vector<KronTask> kron;
        std::vector<TruncTask> tt;
        std::vector<LeafTruncTask> lt;
        int64_t vrow = 0, aoff = 0, gel = 0;
        int smem_n = 0, smem_l = 0;
        for (int64_t a = a0; a < a1; ++a) {
            if (leaf_[a]) {
                LeafTruncTask t{};
                t.z = offZ_[pass][a];
                t.p = offP_[a];
                t.r = offR_[a];
                t.q = offQ_[pass][a];
                t.c = offC_[pass][a];
                t.sig = offSig_[pass][a];
                t.rz = rZ_[pass][a];
                t.rt = rR_[a];
                t.n = rows_[a];
                t.qld = (int32_t)ldQ_[pass][a];
                t.up = offUp_[pass][a];
                t.a = (int32_t)a;
                smem_l = std::max(smem_l, std::min(t.rt, 64));
                lt.push_back(t);
                work_[K_TRUNCATE] += 8.0 * t.rt * t.rt * t.rz + 8.0 * t.n * t.rt * t.rt + 8.0 * t.rt * t.rt * kk;
                continue;
            }
            TruncTask tk{};
            tk.leaf = 0;
            tk.a = (int32_t)a;
            tk.rz = rZ_[pass][a];
            tk.z = offZ_[pass][a];
            tk.q = offQ_[pass][a];
            tk.qld = (int32_t)ldQ_[pass][a];
            tk.c = offC_[pass][a];
            tk.sig = offSig_[pass][a];
            int32_t s0 = sons_[0][a], s1 = sons_[1][a];
            int32_t k0 = rank_[pass][s0], k1 = rank_[pass][s1];
            tk.rows = k0 + k1;
            tk.vsrc = vrow * kk;
            if (k0) kron.push_back(KronTask{offC_[pass][s0], offE_[a], vrow * kk, k0, 0});
            if (k1) kron.push_back(KronTask{offC_[pass][s1], offE_[a] + 3 * m_ * m_, (vrow + k0) * kk, k1, 0});
            vrow += k0 + k1;
            smem_n = std::max(smem_n, std::min(tk.rows, 64));
            tt.push_back(tk);
            // A = V Z^* and M = A A^* (the Jacobi sweeps and C = Q^* V are not counted)
            work_[K_TRUNCATE] += 8.0 * tk.rows * tk.rz * kk + 8.0 * tk.rows * tk.rows * tk.rz;
        }
        for (auto& t : lt) {
            t.scr = gel;
            if (t.rt > smem_l) gel += eig_global_elems(t.rt);
        }
        // scratch per task: A (rows x rz, working precision) and, when rows > smem_n, a
        // global FP64 Jacobi slot
        int64_t goff = 0;
        for (auto& tk : tt) {
            tk.ascratch = aoff;
            aoff += ((int64_t)tk.rows * std::max(tk.rz, 1) + 3) & ~int64_t(3);
            tk.gslot = goff;
            if (tk.rows > smem_n) goff += eig_global_elems(tk.rows);
        }
        vhat.reserve(std::max<int64_t>(vrow * kk, 1));
        ascr.reserve(std::max<int64_t>(aoff, 1));
        gscr.reserve(std::max<int64_t>(goff, 1));
        lscr.reserve(std::max<int64_t>(gel, 1));
        if (!lt.empty()) {
            DBuf<LeafTruncTask> d;
            upload_vec(d, lt, s);
            const size_t smem = eig_smem_bytes(smem_l);
            auto kern = bp_.svd_fp64 ? k_trunc_leaf<T, true> : k_trunc_leaf<T, false>;
            ensure_smem(reinterpret_cast<const void*>(kern), smem);
            ev_.begin(K_TRUNCATE, s);
            kern<<<(unsigned)lt.size(), kThreads, smem, s>>>(d.p, kk, Z_[pass].p, pass == 0 ? P_.p : Pcol(),
                                                              pass == 0 ? R_.p : Rcol(), lscr.p, smem_l,
                                                              bp_.eps, bp_.rank_rule, Q_[pass].p, Cd_[pass].p, Ct,
                                                              sig_[pass].p, rank_d_[pass].p, Up_[pass].p, err_.p);
            ev_.end(s);
            DH2_CHECK_LAUNCH("k_trunc_leaf");
        }
        if (!kron.empty()) {
            DBuf<KronTask> d;
            upload_vec(d, kron, s);
            size_t smem = (2 * (size_t)kk + 3 * m_ * m_) * sizeof(cx<T>);
            ev_.begin(K_KRON, s);
            k_kron<T, T, T, T><<<(unsigned)kron.size(), kThreads, smem, s>>>(d.p, m_, Ct, E_.p, vhat.p);
            ev_.end(s);
            DH2_CHECK_LAUNCH("k_kron");
        }
        if (!tt.empty()) {
            DBuf<TruncTask> d;
            upload_vec(d, tt, s);
            size_t smem = eig_smem_bytes(smem_n);
            auto kern = bp_.svd_fp64 ? k_truncate<T, true> : k_truncate<T, false>;
            ensure_smem(reinterpret_cast<const void*>(kern), smem);
            ev_.begin(K_TRUNCATE, s);
            kern<<<(unsigned)tt.size(), kThreads, smem, s>>>(d.p, kk, vhat.p, Z_[pass].p, ascr.p, gscr.p, smem_n,
                                                              bp_.eps, bp_.rank_rule, Q_[pass].p, Cd_[pass].p, Ct,
                                                              sig_[pass].p, rank_d_[pass].p, err_.p);
            ev_.end(s);
            DH2_CHECK_LAUNCH("k_truncate");
        }
        std::vector<int32_t> rk(a1 - a0);
        DH2_CHECK_CUDA(cudaMemcpyAsync(rk.data(), rank_d_[pass].p + a0, (a1 - a0) * sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, s));
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int64_t a = a0; a < a1; ++a) rank_[pass][a] = rk[a - a0];
        const unsigned e = read_scalar(err_.p, s);
        if (e & ~ERR_RANK_CAP)
            throw Error{DH2_ENUMERIC, "non-finite value in truncation (code " + std::to_string(e) + ")"};
        if (e & ERR_RANK_CAP) return false;
    }
    return true;
}

// ----------------------------------------------------------------------------- projection

template <class T>
template <int NT>
void Num<T>::launch_project_tc(const std::vector<ProjTask>& tasks, cudaStream_t s) {
    if (tasks.empty()) return;
    if constexpr (std::is_same<T, float>::value) {
        DBuf<ProjTask> d;
        upload_vec(d, tasks, s);
        const size_t smem = 128 + 2 * 256 * sizeof(float4) + TcTile<NT>::kOperandBytes;
        auto kern = k_project_tc<NT>;
        ensure_smem(reinterpret_cast<const void*>(kern), smem);
        kern<<<(unsigned)tasks.size(), kThreads, smem, s>>>(d.p, st_.adm_t.p, st_.adm_s.p, st_.adm_c.p, tc_level_.p,
                                                          st_.dir_off_d.p, st_.dirs.p, nodes_.p, m_, bp_.kappa,
                                                          Ct_[0].p, Ct_[1].p, St_.p, err_.p);
        DH2_CHECK_LAUNCH("k_project_tc");
    }
}

template <class T>
void Num<T>::project(cudaStream_t s) {
    const auto& h = hs_;
    const int64_t nb = (int64_t)h.adm_t.size();
    std::vector<ProjTask> pt(nb);
    // S~ storage in row-list order: the couplings of one row pair are contiguous
    st_off_.assign(nb + 1, 0);
    {
        int64_t o = 0;
        for (int64_t a = 0; a < na_; ++a) {
            int32_t tc = h.tc_base[h.a_t[a]] + h.a_c[a];
            for (int32_t e = h.row_ptr[tc]; e < h.row_ptr[tc + 1]; ++e) {
                int32_t b = h.row_idx[e];
                int32_t c = h.adm_c[b];
                st_off_[b] = o;
                o += (int64_t)rank_[0][h.pair_of(h.adm_t[b], c)] * rank_[1][h.pair_of(h.adm_s[b], c)];
            }
        }
        st_off_[nb] = o;
    }
    int64_t off = 0;
    for (int64_t b = 0; b < nb; ++b) {
        int32_t c = h.adm_c[b];
        int32_t at = h.pair_of(h.adm_t[b], c), as = h.pair_of(h.adm_s[b], c);
        ProjTask p{};
        p.b = (int32_t)b;
        p.kt = rank_[0][at];
        p.ks = rank_[1][as];
        p.crow = offC_[0][at];
        p.ccol = offC_[1][as];
        p.dst = st_off_[b];
        p.leafpair = leaf_[at] && leaf_[as] && kstore_;
        if (p.leafpair) {
            p.koff = offK_[b];
            p.upt = offUp_[0][at];
            p.ups = offUp_[1][as];
            p.rt = rR_[at];
            p.rs = rR_[as];
            p.ldt = (int32_t)ldQ_[0][at];
            p.lds = (int32_t)ldQ_[1][as];
        }
        off += (int64_t)p.kt * p.ks;
        pt[b] = p;
        if (p.kt && p.ks)
            work_[K_PROJECT] += p.leafpair ? 8.0 * p.kt * p.rt * p.rs + 8.0 * p.kt * p.rs * p.ks
                                           : kEvalFlops * k_ * k_ + 8.0 * p.kt * k_ * k_ + 8.0 * p.kt * k_ * p.ks;
    }
    info.coupling_entries = off;
    St_.alloc(std::max<int64_t>(off, 1));
    if (nb == 0) return;
    if constexpr (std::is_same<T, float>::value) {
        if (bp_.tensor_cores && k_ <= 256) {
            // blocks whose clusters are not both leaves: tensor-core tiles by k_t (with k > 128
            // only k_t <= 64, see total_weights)
            std::vector<ProjTask> rest, cls[3];
            for (const ProjTask& p : pt) {
                const int c = p.kt <= 32 ? 0 : p.kt <= 64 ? 1 : 2;
                if (p.leafpair || p.kt == 0 || p.ks == 0 || (c == 2 && k_ > 128)) rest.push_back(p);
                else cls[c].push_back(p);
            }
            ev_.begin(K_PROJECT, s);
            launch_project_tc<64>(cls[0], s);
            launch_project_tc<128>(cls[1], s);
            launch_project_tc<256>(cls[2], s);
            ev_.end(s);
            pt.swap(rest);
        }
    }
    const int64_t np_ = (int64_t)pt.size();
    if (np_ == 0) {
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        return;
    }
    DBuf<ProjTask> d;
    upload_vec(d, pt, s);
    const int64_t grid = std::min<int64_t>(np_, 152 * 8);
    DBuf<cx<T>> scratch((size_t)grid * k_ * k_);
    const cx<T>* Crow;
    const cx<T>* Ccol;
    if constexpr (std::is_same<T, float>::value) {
        Crow = Ct_[0].p;
        Ccol = Ct_[1].p;
    } else {
        Crow = reinterpret_cast<const cx<T>*>(Cd_[0].p);
        Ccol = reinterpret_cast<const cx<T>*>(Cd_[1].p);
    }
    const size_t smem = sgen_smem_bytes<T>(m_);
    ev_.begin(K_PROJECT, s);
    k_project<T><<<(unsigned)grid, kThreads, smem, s>>>(d.p, np_, st_.adm_t.p, st_.adm_s.p, st_.adm_c.p,
                                                        tc_level_.p, st_.dir_off_d.p, st_.dirs.p, nodes_.p, m_,
                                                        bp_.kappa, Crow, Ccol, K_.p, Up_[0].p, Up_[1].p, scratch.p,
                                                        St_.p);
    ev_.end(s);
    DH2_CHECK_LAUNCH("k_project");
    DH2_CHECK_CUDA(cudaStreamSynchronize(s));
}

// the projection stage, then its device error check (a tensor-core wait that gave up leaves
// S~ partly written)
template <class T>
void Num<T>::project_checked(cudaStream_t s) {
    project(s);
    inject_fault(s);
    check_err(s, "projection");
    K_.release();   // read by nothing after the projection
    kb_hold_.release();
}

// ----------------------------------------------------------------------------- matvec plan

template <class T>
void Num<T>::plan_matvec(cudaStream_t s) {
    const auto& h = hs_;
    std::vector<int64_t> xh_off(na_ + 1), yh_off(na_ + 1);
    for (int64_t a = 0; a < na_; ++a) {
        xh_off[a + 1] = xh_off[a] + rank_[1][a];
        yh_off[a + 1] = yh_off[a] + rank_[0][a];
    }
    xt_.alloc(std::max<int64_t>(n_, 1));
    xh_.alloc(std::max<int64_t>(xh_off[na_], 1));
    yh_.alloc(std::max<int64_t>(yh_off[na_], 1));
    int64_t basis_entries = 0;
    // forward transform
    std::vector<FwdLeaf> fl;
    std::vector<FwdUp> fu;
    fwd_up_level_counts_.assign(h.depth + 1, 0);
    for (int l = h.depth; l >= 0; --l) {
        for (int64_t a = h.alevel_start[l]; a < h.alevel_start[l + 1]; ++a) {
            const int k = rank_[1][a];
            if (leaf_[a]) {
                basis_entries += (int64_t)rows_[a] * k;
                if (k) fl.push_back(FwdLeaf{offQ_[1][a], xh_off[a], (int32_t)ldQ_[1][a], rows_[a], h.offset[h.a_t[a]], k});
            } else {
                int32_t s0 = sons_[0][a], s1 = sons_[1][a];
                basis_entries += (int64_t)(rank_[1][s0] + rank_[1][s1]) * k;
                if (k) {
                    fu.push_back(FwdUp{offQ_[1][a], xh_off[a], xh_off[s0], xh_off[s1], (int32_t)ldQ_[1][a],
                                       rank_[1][s0], rank_[1][s1], k});
                    fwd_up_level_counts_[l]++;
                }
            }
        }
    }
    n_fwd_leaf_ = (int64_t)fl.size();
    upload_vec(fwd_leaf_, fl, s);
    upload_vec(fwd_up_, fu, s);
    // couplings: S~ offsets from the projection (row-list order)
    const std::vector<int64_t>& st_off = st_off_;
    std::vector<int32_t> cptr(na_ + 1, 0);
    std::vector<Coup> items;
    for (int64_t a = 0; a < na_; ++a) {
        int32_t t = h.a_t[a], c = h.a_c[a], tc = h.tc_base[t] + c;
        for (int32_t e = h.row_ptr[tc]; e < h.row_ptr[tc + 1]; ++e) {
            int32_t b = h.row_idx[e];
            int32_t as = h.pair_of(h.adm_s[b], c);
            if (rank_[0][a] == 0 || rank_[1][as] == 0) continue;
            items.push_back(Coup{st_off[b], xh_off[as], rank_[0][a], rank_[1][as]});
        }
        cptr[a + 1] = (int32_t)items.size();
    }
    upload_vec(coup_ptr_, cptr, s);
    upload_vec(coup_, items, s);
    {   // tiles of the coupling products: runs of whole blocks of at most kCoupTile bytes per row pair
        const int64_t cap = (int64_t)(kCoupTile / sizeof(cx<T>));
        std::vector<CoupTile> tiles;
        std::vector<CoupRow> crow;
        std::vector<int64_t> first;
        int64_t out = 0, entries = 0;
        for (int64_t a = 0; a < na_; ++a) {
            const int32_t e_beg = cptr[a], e_end = cptr[a + 1], kt = rank_[0][a];
            if (kt == 0) continue;
            const int64_t t0 = (int64_t)tiles.size(), out0 = out;
            int32_t e = e_beg;
            while (e < e_end) {
                int64_t tot = 0;
                int32_t e1 = e;
                while (e1 < e_end) {
                    const int64_t sz = (int64_t)kt * items[e1].ks;
                    if (e1 > e && tot + sz > cap) break;
                    tot += sz;
                    ++e1;
                }
                tiles.push_back(CoupTile{e, e1, kt, 0, out});
                out += kt;
                e = e1;
            }
            crow.push_back(CoupRow{yh_off[a], out0, (int32_t)((int64_t)tiles.size() - t0), kt});
            first.push_back(entries);
            entries += kt;
        }
        n_coup_tiles_ = (int64_t)tiles.size();
        n_coup_rows_ = (int64_t)crow.size();
        n_coup_entries_ = entries;
        upload_vec(coup_tiles_, tiles, s);
        upload_vec(coup_rows_, crow, s);
        upload_vec(coup_first_, first, s);
        coup_psum_.alloc(std::max<int64_t>(out, 1));
    }
    std::vector<int32_t> kr(rank_[0].begin(), rank_[0].end());
    upload_vec(krow_d_, kr, s);
    std::vector<int64_t> yo(yh_off.begin(), yh_off.end() - 1);
    upload_vec(yh_off_, yo, s);
    // backward transform, top-down
    std::vector<int32_t> bp, bptr{0};
    std::vector<Bwd> bitems;
    bwd_level_counts_.assign(h.depth + 1, 0);
    for (int l = 1; l <= h.depth; ++l) {
        for (int64_t a = h.alevel_start[l]; a < h.alevel_start[l + 1]; ++a) {
            if (rank_[0][a] == 0) continue;
            bool any = false;
            for (auto& pr : parents_[a]) {
                int32_t ap = pr.first;
                if (rank_[0][ap] == 0) continue;
                int64_t rowoff = pr.second == 0 ? 0 : rank_[0][sons_[0][ap]];
                bitems.push_back(Bwd{offQ_[0][ap] + rowoff * ldQ_[0][ap], yh_off[ap], (int32_t)ldQ_[0][ap], rank_[0][ap]});
                any = true;
            }
            if (any) {
                bp.push_back((int32_t)a);
                bptr.push_back((int32_t)bitems.size());
                bwd_level_counts_[l]++;
            }
        }
        if (!leaf_.empty()) {
            for (int64_t a = h.alevel_start[l - 1]; a < h.alevel_start[l]; ++a)
                if (!leaf_[a]) basis_entries += 0;
        }
    }
    upload_vec(bwd_pairs_, bp, s);
    upload_vec(bwd_ptr_, bptr, s);
    upload_vec(bwd_, bitems, s);
    // row basis storage (leaf Q and transfers F)
    for (int64_t a = 0; a < na_; ++a) {
        if (leaf_[a])
            basis_entries += (int64_t)rows_[a] * rank_[0][a];
        else
            basis_entries += (int64_t)(rank_[0][sons_[0][a]] + rank_[0][sons_[1][a]]) * rank_[0][a];
    }
    info.basis_entries = basis_entries;
    // leaf output: far-field Q items and nearfield segments per leaf
    std::vector<int32_t> leaf_index(h.nc, -1);
    for (size_t i = 0; i < leaf_order_.size(); ++i) leaf_index[leaf_order_[i]] = (int32_t)i;
    std::vector<std::vector<LeafQ>> per_leaf(leaf_order_.size());
    for (int64_t a = 0; a < na_; ++a) {
        if (!leaf_[a] || rank_[0][a] == 0) continue;
        per_leaf[leaf_index[h.a_t[a]]].push_back(LeafQ{offQ_[0][a], yh_off[a], (int32_t)ldQ_[0][a], rank_[0][a]});
    }
    std::vector<LeafOut> lo;
    std::vector<LeafQ> lq;
    std::vector<LeafSeg> ls;
    for (size_t i = 0; i < leaf_order_.size(); ++i) {
        LeafOut o{};
        o.off = h.offset[leaf_order_[i]];
        o.rows = h.size[leaf_order_[i]];
        o.qbeg = (int32_t)lq.size();
        for (auto& q : per_leaf[i]) lq.push_back(q);
        o.qend = (int32_t)lq.size();
        o.sbeg = (int32_t)ls.size();
        for (auto& sg : leaf_segs_[i]) ls.push_back(LeafSeg{sg.poff, sg.ld, sg.coff, sg.cols, 0});
        o.send = (int32_t)ls.size();
        lo.push_back(o);
    }
    upload_vec(leaf_out_, lo, s);
    upload_vec(leaf_q_, lq, s);
    upload_vec(leaf_seg_, ls, s);
    std::vector<LeafOut2> lo2;
    for (size_t i = 0; i < leaf_order_.size(); ++i) {
        LeafOut2 o{};
        o.poff = leaf_poff_[i];
        o.coff = leaf_coff_[i];
        o.off = lo[i].off;
        o.rows = lo[i].rows;
        o.ld = leaf_ld_[i];
        o.qbeg = lo[i].qbeg;
        o.qend = lo[i].qend;
        lo2.push_back(o);
    }
    // nearfield parts of the graph product: every panel cut into kNearChunk-column chunks
    std::vector<NearPart> np;
    int64_t pofs = 0;
    for (auto& o : lo2) {
        o.nbeg = (int32_t)np.size();
        for (int32_t c0 = 0; c0 < o.ld; c0 += kNearChunk) {
            NearPart pt{};
            pt.poff = o.poff + c0;
            pt.coff = o.coff + c0;
            pt.pofs = pofs;
            pt.rows = o.rows;
            pt.ld = o.ld;
            pt.w = std::min(kNearChunk, o.ld - c0);
            np.push_back(pt);
            pofs += o.rows;
        }
        o.nend = (int32_t)np.size();
    }
    n_near_parts_ = (int64_t)np.size();
    upload_vec(near_parts_, np, s);
    near_pbuf_.alloc(std::max<int64_t>(pofs, 1));
    upload_vec(leaf_out2_, lo2, s);
    const int64_t cs = sizeof(cx<T>);
    info.matvec_bytes = (info.near_entries + info.coupling_entries + info.basis_entries) * cs +
                        2 * n_ * cs + 2 * (xh_off[na_] + yh_off[na_]) * cs;
    // ranks summary
    int64_t cnt = 0;
    double sr = 0, sc_ = 0;
    for (int64_t a = 0; a < na_; ++a) {
        info.max_rank_row = std::max(info.max_rank_row, rank_[0][a]);
        info.max_rank_col = std::max(info.max_rank_col, rank_[1][a]);
        sr += rank_[0][a];
        sc_ += rank_[1][a];
        ++cnt;
    }
    info.mean_rank_row = cnt ? sr / cnt : 0;
    info.mean_rank_col = cnt ? sc_ / cnt : 0;
    DH2_CHECK_CUDA(cudaStreamSynchronize(s));
}

// ----------------------------------------------------------------------------- build

template <class T>
void Num<T>::build(cudaStream_t s) {
    StageTimer tm(s);
    err_.alloc(1);
    err_.zero(s);
    layout();
    setup_symmetry(s);
    info.symmetric = sym_ ? 1 : 0;
    tm.begin(ST_ANALYTIC);
    analytic(s);
    tm.end(ST_ANALYTIC);
    // The nearfield (read only by the matvec plan) is planned on a host thread and computed on
    // its own stream while the recompression runs; it starts after the analytic stage (the
    // double layer's normals) and the matvec plan waits for it.
    int dev = 0;
    DH2_CHECK_CUDA(cudaGetDevice(&dev));
    if (!near_stream_) DH2_CHECK_CUDA(cudaStreamCreateWithFlags(&near_stream_, cudaStreamNonBlocking));
    struct Events {   // destroyed on every path out of the build
        cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } evs;
    DH2_CHECK_CUDA(cudaEventCreateWithFlags(&evs.e[0], cudaEventDisableTiming));
    DH2_CHECK_CUDA(cudaEventCreate(&evs.e[1]));
    DH2_CHECK_CUDA(cudaEventCreate(&evs.e[2]));
    cudaEvent_t nf_fork = evs.e[0], nf_t0 = evs.e[1], nf_t1 = evs.e[2];
    DH2_CHECK_CUDA(cudaEventRecord(nf_fork, s));
    DH2_CHECK_CUDA(cudaStreamWaitEvent(near_stream_, nf_fork, 0));
    EventLog nf_ev;
    std::exception_ptr nf_err;
    {
        struct Joiner {   // joined on every path out of this scope
            std::thread t;
            ~Joiner() {
                if (t.joinable()) t.join();
            }
        } nf;
        nf.t = std::thread([&] {
            try {
                DH2_CHECK_CUDA(cudaSetDevice(dev));
                AllocScope scope(near_stream_);
                DH2_CHECK_CUDA(cudaEventRecord(nf_t0, near_stream_));
                nearfield(near_stream_, nf_ev);
                DH2_CHECK_CUDA(cudaEventRecord(nf_t1, near_stream_));
            } catch (...) {
                nf_err = std::current_exception();
            }
        });
        build_recompression(s, tm);
        nf.t.join();
    }
    if (nf_err) std::rethrow_exception(nf_err);
    DH2_CHECK_CUDA(cudaEventRecord(nf_fork, near_stream_));
    DH2_CHECK_CUDA(cudaStreamWaitEvent(s, nf_fork, 0));
    tm.begin(ST_MATVEC_PLAN);
    plan_matvec(s);
    tm.end(ST_MATVEC_PLAN);
    tm.collect(info.stage_ms);
    {
        float ms = 0;
        DH2_CHECK_CUDA(cudaEventElapsedTime(&ms, nf_t0, nf_t1));
        info.stage_ms[ST_NEARFIELD] += ms;
    }
    ev_.recs.insert(ev_.recs.end(), nf_ev.recs.begin(), nf_ev.recs.end());
    nf_ev.recs.clear();
    finish_info();
}

// The recompression stages of the build (Section 3.2) and the projection, on stream s.
template <class T>
void Num<T>::build_recompression(cudaStream_t s, StageTimer& tm) {
    tm.begin(ST_BASIS_WEIGHTS);
    basis_weights(s);
    tm.end(ST_BASIS_WEIGHTS);
    tm.begin(ST_TOTAL_WEIGHTS_ROW);
    total_weights(0, s);
    tm.end(ST_TOTAL_WEIGHTS_ROW);
    tm.begin(ST_TOTAL_WEIGHTS_COL);
    total_weights(1, s);
    tm.end(ST_TOTAL_WEIGHTS_COL);
    tm.begin(ST_TRUNCATE_ROW);
    truncate(0, s);
    tm.end(ST_TRUNCATE_ROW);
    tm.begin(ST_TRUNCATE_COL);
    truncate(1, s);
    tm.end(ST_TRUNCATE_COL);
    if (bp_.direct) {   // read by nothing after the truncation (the projection uses C, U' and K_b)
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        V_.release();
        W_.release();
        E_.release();
        R_.release();
        P_.release();
        RW_.release();
        PW_.release();
        Z_[0].release();
        Z_[1].release();
    }
    tm.begin(ST_PROJECT);
    project_checked(s);
    tm.end(ST_PROJECT);
}

// kernel times and work of the finished build
template <class T>
void Num<T>::finish_info() {
    ev_.collect(info);
    const int32_t w32 = std::is_same<T, float>::value ? W_FLOP32 : W_FLOP64;
    const int32_t wqr = (std::is_same<T, double>::value || bp_.qr_fp64) ? W_FLOP64 : W_FLOP32;
    for (int i = 0; i < K_COUNT; ++i) info.kernel_work[i] = work_[i];
    info.kernel_work[K_NEARFIELD] = 9.0 * kEvalFlops * info.near_entries;
    info.kernel_work_kind[K_NEARFIELD] = w32;
    info.kernel_work_kind[K_KRON] = w32;
    info.kernel_work_kind[K_STACK_BLOCKS] = w32;
    info.kernel_work_kind[K_TSQR] = wqr;
    info.kernel_work_kind[K_TRUNCATE] = (std::is_same<T, double>::value || bp_.svd_fp64) ? W_FLOP64 : W_FLOP32;
    info.kernel_work_kind[K_LEAF_ORTH] = wqr;
    info.kernel_work_kind[K_TSQR_NARROW] = info.kernel_work_kind[K_TSQR];
    if (gram_slices()) {   // the Gram tiles ran on the tensor cores: their BF16 work
        info.kernel_work[K_TSQR_NARROW] = gram_mma_flops_[0];
        info.kernel_work[K_TSQR] = gram_mma_flops_[1];
        info.kernel_work_kind[K_TSQR_NARROW] = W_FLOP_BF16;
        info.kernel_work_kind[K_TSQR] = W_FLOP_BF16;
    }
    info.kernel_work_kind[K_WQR_CHOL] = W_FLOP64;
    info.kernel_work_kind[K_PROJECT] = w32;
    // matvec leaf kernel: nearfield panels + leaf row bases streamed once, x and y once
    int64_t qleaf = 0;
    for (int64_t a = 0; a < na_; ++a)
        if (leaf_[a]) qleaf += (int64_t)rows_[a] * rank_[0][a];
    info.kernel_work[K_MV_LEAF_OUT] = (double)(info.near_entries + qleaf + 2 * n_) * sizeof(cx<T>);
    info.kernel_work_kind[K_MV_LEAF_OUT] = W_BYTES;
}

// ----------------------------------------------------------------------------- matvec

// y = G~ x.  Without per-kernel timing the product runs as a CUDA graph: its ~40 launches
// (one per tree level for the transforms) are captured once per precision, on an internal
// stream, against internal copies of x and y, and replayed on the caller's stream between
// two device copies of n values; the graph's parameters never change.
template <class T>
void Num<T>::matvec(const void* x, void* y, int dtype, cudaStream_t s) {
    if (timing_on_) {
        launch_matvec(x, y, dtype, s);
        return;
    }
    const int di = dtype == DH2_C64 ? 0 : 1;
    const size_t bytes = (size_t)n_ * (dtype == DH2_C64 ? sizeof(cx<float>) : sizeof(cx<double>));
    MatvecGraph& mg = graph_[di];
    if (!mg.exec) {
        mg.x.alloc(bytes);
        mg.y.alloc(bytes);
        if (!capture_stream_) DH2_CHECK_CUDA(cudaStreamCreateWithFlags(&capture_stream_, cudaStreamNonBlocking));
        if (!side_stream_) {
            DH2_CHECK_CUDA(cudaStreamCreateWithFlags(&side_stream_, cudaStreamNonBlocking));
            DH2_CHECK_CUDA(cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming));
            DH2_CHECK_CUDA(cudaEventCreateWithFlags(&join_ev_, cudaEventDisableTiming));
        }
        cudaGraph_t graph = nullptr;
        DH2_CHECK_CUDA(cudaStreamBeginCapture(capture_stream_, cudaStreamCaptureModeThreadLocal));
        try {
            launch_matvec(mg.x.p, mg.y.p, dtype, capture_stream_, true);
        } catch (...) {
            cudaStreamEndCapture(capture_stream_, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        DH2_CHECK_CUDA(cudaStreamEndCapture(capture_stream_, &graph));
        size_t nodes = 0;   // every node is one captured kernel launch
        cudaGraphGetNodes(graph, nullptr, &nodes);
        mg.nodes = (int64_t)nodes;
        uncount_launches(mg.nodes);   // counted when captured, not launched
        const cudaError_t e = cudaGraphInstantiate(&mg.exec, graph, 0);
        cudaGraphDestroy(graph);
        DH2_CHECK_CUDA(e);
    }
    DH2_CHECK_CUDA(cudaMemcpyAsync(mg.x.p, x, bytes, cudaMemcpyDeviceToDevice, s));
    DH2_CHECK_CUDA(cudaGraphLaunch(mg.exec, s));
    DH2_CHECK_CUDA(cudaMemcpyAsync(y, mg.y.p, bytes, cudaMemcpyDeviceToDevice, s));
    count_launches(mg.nodes);
}

// split = true (graph capture only): the nearfield part of the output runs on a side branch
// that forks after the gather (k_near_part, panel column chunks) and joins before the
// leaf-basis part, which adds the chunks' partial sums in a fixed order and writes y.
template <class T>
void Num<T>::launch_matvec(const void* x, void* y, int dtype, cudaStream_t s, bool split) {
    const unsigned g = grid_for(n_, kThreads);
    if (dtype == DH2_C64) {
        if (timing_on_) ev_.begin(K_MV_GATHER, s);
        k_gather<T, float><<<g, kThreads, 0, s>>>(tr_.perm.p, n_, (const cx<float>*)x, xt_.p);
        if (timing_on_) ev_.end(s);
    }
    else {
        if (timing_on_) ev_.begin(K_MV_GATHER, s);
        k_gather<T, double><<<g, kThreads, 0, s>>>(tr_.perm.p, n_, (const cx<double>*)x, xt_.p);
        if (timing_on_) ev_.end(s);
    }
    DH2_CHECK_LAUNCH("k_gather");
    if (split && n_leaves_) {
        DH2_CHECK_CUDA(cudaEventRecord(fork_ev_, s));
        DH2_CHECK_CUDA(cudaStreamWaitEvent(side_stream_, fork_ev_, 0));
        if (n_near_parts_) {
            k_near_part<T><<<(unsigned)n_near_parts_, 256, 0, side_stream_>>>(near_parts_.p, colidx_.p, near_.p,
                                                                           xt_.p, near_pbuf_.p);
            DH2_CHECK_LAUNCH("k_near_part");
        }
        DH2_CHECK_CUDA(cudaEventRecord(join_ev_, side_stream_));
    }
    constexpr int WPB = 8;   // warps per CTA of the transform kernels
    if (n_fwd_leaf_) {
        if (timing_on_) ev_.begin(K_MV_FORWARD, s);
        k_fwd_leaf<T><<<grid_for(n_fwd_leaf_, WPB), WPB * 32, 0, s>>>(fwd_leaf_.p, n_fwd_leaf_, Q_[1].p, xt_.p, xh_.p);
        if (timing_on_) ev_.end(s);
        DH2_CHECK_LAUNCH("k_fwd_leaf");
    }
    int64_t off = 0;
    for (int l = hs_.depth; l >= 0; --l) {
        int64_t cnt = fwd_up_level_counts_[l];
        if (cnt) {
            if (timing_on_) ev_.begin(K_MV_FORWARD, s);
            k_fwd_up<T><<<grid_for(cnt, WPB), WPB * 32, 0, s>>>(fwd_up_.p + off, cnt, Q_[1].p, xh_.p);
            if (timing_on_) ev_.end(s);
            DH2_CHECK_LAUNCH("k_fwd_up");
        }
        off += cnt;
    }
    if (na_) {
        if (timing_on_) ev_.begin(K_MV_COUPLING, s);
        launch_coupling(xh_.p, yh_.p, s);
        if (timing_on_) ev_.end(s);
    }
    off = 0;
    for (int l = 1; l <= hs_.depth; ++l) {
        int64_t cnt = bwd_level_counts_[l];
        if (cnt) {
            if (timing_on_) ev_.begin(K_MV_BACKWARD, s);
            k_backward<T><<<grid_for(cnt, WPB), WPB * 32, 0, s>>>(bwd_pairs_.p + off, bwd_ptr_.p + off, bwd_.p,
                                                                  yh_off_.p, krow_d_.p, cnt, Q_[0].p, yh_.p);
            if (timing_on_) ev_.end(s);
            DH2_CHECK_LAUNCH("k_backward");
        }
        off += cnt;
    }
    if (split && n_leaves_) {
        DH2_CHECK_CUDA(cudaStreamWaitEvent(s, join_ev_, 0));
        if (dtype == DH2_C64)
            k_leaf_out2<T, float, 2><<<(unsigned)n_leaves_, 256, 0, s>>>(
                leaf_out2_.p, leaf_q_.p, colidx_.p, Q_[0].p, yh_.p, near_.p, xt_.p, tr_.perm.p, (cx<float>*)y,
                near_parts_.p, near_pbuf_.p);
        else
            k_leaf_out2<T, double, 2><<<(unsigned)n_leaves_, 256, 0, s>>>(
                leaf_out2_.p, leaf_q_.p, colidx_.p, Q_[0].p, yh_.p, near_.p, xt_.p, tr_.perm.p, (cx<double>*)y,
                near_parts_.p, near_pbuf_.p);
        DH2_CHECK_LAUNCH("k_leaf_out2 (leaf bases)");
    } else if (n_leaves_ && timing_on_ && n_near_parts_) {
        // timed products run the graph's decomposition serially: the nearfield in panel column
        // parts (balanced over the SMs), then the leaf bases plus the parts' sums; both launches
        // count as the leaf output
        ev_.begin(K_MV_LEAF_OUT, s);
        k_near_part<T><<<(unsigned)n_near_parts_, 256, 0, s>>>(near_parts_.p, colidx_.p, near_.p, xt_.p,
                                                                near_pbuf_.p);
        ev_.end(s);
        DH2_CHECK_LAUNCH("k_near_part");
        ev_.begin(K_MV_LEAF_OUT, s);
        if (dtype == DH2_C64)
            k_leaf_out2<T, float, 2><<<(unsigned)n_leaves_, 256, 0, s>>>(
                leaf_out2_.p, leaf_q_.p, colidx_.p, Q_[0].p, yh_.p, near_.p, xt_.p, tr_.perm.p, (cx<float>*)y,
                near_parts_.p, near_pbuf_.p);
        else
            k_leaf_out2<T, double, 2><<<(unsigned)n_leaves_, 256, 0, s>>>(
                leaf_out2_.p, leaf_q_.p, colidx_.p, Q_[0].p, yh_.p, near_.p, xt_.p, tr_.perm.p, (cx<double>*)y,
                near_parts_.p, near_pbuf_.p);
        ev_.end(s);
        DH2_CHECK_LAUNCH("k_leaf_out2 (leaf bases)");
    } else if (n_leaves_) {
        if (dtype == DH2_C64) {
            if (timing_on_) ev_.begin(K_MV_LEAF_OUT, s);
            k_leaf_out2<T, float, 0><<<(unsigned)n_leaves_, 256, 0, s>>>(leaf_out2_.p, leaf_q_.p, colidx_.p, Q_[0].p,
                                                                    yh_.p, near_.p, xt_.p, tr_.perm.p, (cx<float>*)y);
            if (timing_on_) ev_.end(s);
        }
        else {
            if (timing_on_) ev_.begin(K_MV_LEAF_OUT, s);
            k_leaf_out2<T, double, 0><<<(unsigned)n_leaves_, 256, 0, s>>>(leaf_out2_.p, leaf_q_.p, colidx_.p, Q_[0].p,
                                                                     yh_.p, near_.p, xt_.p, tr_.perm.p, (cx<double>*)y);
            if (timing_on_) ev_.end(s);
        }
        DH2_CHECK_LAUNCH("k_leaf_out");
    }
    if (timing_on_) ev_.collect(info);
}


// ----------------------------------------------------------------------------- allocation-free matvec
//
// Some callers cannot call cudaMalloc at the point where they need a product:
// code that records work into a CUDA graph while another framework owns every
// device allocation, host threads running inside a real-time or interrupt-like
// loop where an allocator call may block, or runtimes that hand this library a
// fixed memory budget.  dh2_matvec_noalloc serves them: it runs the same kernels
// as dh2_matvec, but its scratch (the permuted input and the basis coefficients
// of the forward and backward transforms) lives in the fixed device array below
// instead of the matrix's own buffers.  The array is a file-scope __device__
// variable: every GPU that loads the library holds its 16 MiB until the process
// exits.  All calls share it and it keeps the last call's contents; every kernel
// writes its part of the scratch before reading it, so nothing needs clearing.
// Two calls whose work overlaps on the GPU (other streams, other host threads)
// race on the array and must be serialised by the caller.

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[128] = {nullptr};

// Device address of g_noalloc_scratch on the current device.  In host code the
// symbol is only a stand-in, so the address comes from cudaGetSymbolAddress,
// once per device, with that device current.
void* noalloc_scratch() {
    int dev = 0;
    DH2_CHECK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) throw Error{DH2_EUNSUPPORTED, "device index out of range"};
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        DH2_CHECK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

template <class T>
void Num<T>::matvec_noalloc(const void* x, void* y, int dtype, cudaStream_t s) {
    const size_t cs = sizeof(cx<T>);
    const size_t bx = align256(std::max<int64_t>(n_, 1) * cs);
    const size_t bxh = align256(xh_.n * cs), byh = align256(yh_.n * cs);
    if (bx + bxh + byh > kNoAllocScratchBytes)
        throw Error{DH2_EINVAL, "dh2_matvec_noalloc: this matrix needs " + std::to_string(bx + bxh + byh) +
                                    " bytes of scratch, more than the fixed " +
                                    std::to_string(kNoAllocScratchBytes) + " bytes"};
    unsigned char* base = static_cast<unsigned char*>(noalloc_scratch());
    cx<T>* xt = reinterpret_cast<cx<T>*>(base);
    cx<T>* xh = reinterpret_cast<cx<T>*>(base + bx);
    cx<T>* yh = reinterpret_cast<cx<T>*>(base + bx + bxh);
    const unsigned g = grid_for(n_, kThreads);
    if (dtype == DH2_C64)
        k_gather<T, float><<<g, kThreads, 0, s>>>(tr_.perm.p, n_, (const cx<float>*)x, xt);
    else
        k_gather<T, double><<<g, kThreads, 0, s>>>(tr_.perm.p, n_, (const cx<double>*)x, xt);
    DH2_CHECK_LAUNCH("k_gather");
    constexpr int WPB = 8;
    if (n_fwd_leaf_) {
        k_fwd_leaf<T><<<grid_for(n_fwd_leaf_, WPB), WPB * 32, 0, s>>>(fwd_leaf_.p, n_fwd_leaf_, Q_[1].p, xt, xh);
        DH2_CHECK_LAUNCH("k_fwd_leaf");
    }
    int64_t off = 0;
    for (int l = hs_.depth; l >= 0; --l) {
        int64_t cnt = fwd_up_level_counts_[l];
        if (cnt) {
            k_fwd_up<T><<<grid_for(cnt, WPB), WPB * 32, 0, s>>>(fwd_up_.p + off, cnt, Q_[1].p, xh);
            DH2_CHECK_LAUNCH("k_fwd_up");
        }
        off += cnt;
    }
    if (na_) {
        launch_coupling(xh, yh, s);
    }
    off = 0;
    for (int l = 1; l <= hs_.depth; ++l) {
        int64_t cnt = bwd_level_counts_[l];
        if (cnt) {
            k_backward<T><<<grid_for(cnt, WPB), WPB * 32, 0, s>>>(bwd_pairs_.p + off, bwd_ptr_.p + off, bwd_.p,
                                                                  yh_off_.p, krow_d_.p, cnt, Q_[0].p, yh);
            DH2_CHECK_LAUNCH("k_backward");
        }
        off += cnt;
    }
    if (n_leaves_) {
        if (dtype == DH2_C64)
            k_leaf_out2<T, float, 0><<<(unsigned)n_leaves_, 256, 0, s>>>(leaf_out2_.p, leaf_q_.p, colidx_.p, Q_[0].p,
                                                                    yh, near_.p, xt, tr_.perm.p, (cx<float>*)y);
        else
            k_leaf_out2<T, double, 0><<<(unsigned)n_leaves_, 256, 0, s>>>(leaf_out2_.p, leaf_q_.p, colidx_.p, Q_[0].p,
                                                                     yh, near_.p, xt, tr_.perm.p, (cx<double>*)y);
        DH2_CHECK_LAUNCH("k_leaf_out");
    }
}

// ----------------------------------------------------------------------------- exports

template <class T>
void Num<T>::export_pair(int which, int64_t tc, double* out, int64_t cap, int32_t* rows, int32_t* cols,
                         cudaStream_t s) {
    *rows = 0;
    *cols = 0;
    if (tc < 0 || tc >= (int64_t)hs_.aidx.size()) throw Error{DH2_EINVAL, "pair index out of range"};
    const int32_t a = hs_.aidx[tc];
    if (a < 0) return;
    const int pass = (which == DH2_X_ZCOL || which == DH2_X_SCOL || which == DH2_X_QCOL || which == DH2_X_CCOL) ? 1 : 0;
    if (bp_.direct && (which == DH2_X_R || which == DH2_X_ZROW || which == DH2_X_ZCOL || which == DH2_X_P ||
                       which == DH2_X_RW || which == DH2_X_PW))
        throw Error{DH2_EUNSUPPORTED, "a direct-recompression build releases R, P and the total weights"};
    int64_t r = 0, c = 0, ld = 0, off = 0;
    const void* src = nullptr;
    bool is_double = std::is_same<T, double>::value, is_real = false;
    const int rowsA = leaf_[a] ? rows_[a] : rank_[pass][sons_[0][a]] + rank_[pass][sons_[1][a]];
    switch (which) {
        case DH2_X_R: r = rR_[a]; c = k_; ld = k_; off = offR_[a]; src = R_.p; break;
        case DH2_X_RW: r = rR_[a]; c = k_; ld = k_; off = offR_[a]; src = Rcol(); break;
        case DH2_X_PW:
            if (!leaf_[a]) return;
            r = rows_[a]; c = rR_[a]; ld = c; off = offP_[a]; src = Pcol(); break;
        case DH2_X_ZROW: case DH2_X_ZCOL:
            r = rZ_[pass][a]; c = zcols(a); ld = c; off = offZ_[pass][a]; src = Z_[pass].p; break;
        case DH2_X_P:
            if (!leaf_[a]) return;
            r = rows_[a]; c = rR_[a]; ld = c; off = offP_[a]; src = P_.p; break;
        case DH2_X_SROW: case DH2_X_SCOL:
            r = 1; c = std::min(rowsA, rZ_[pass][a]); ld = c; off = offSig_[pass][a]; src = sig_[pass].p;
            is_real = true; is_double = true; break;
        case DH2_X_QROW: case DH2_X_QCOL: r = rowsA; c = rank_[pass][a]; ld = ldQ_[pass][a]; off = offQ_[pass][a]; src = Q_[pass].p; break;
        case DH2_X_CROW: case DH2_X_CCOL: r = rank_[pass][a]; c = k_; ld = k_; off = offC_[pass][a]; src = Cd_[pass].p; is_double = true; break;
        default: throw Error{DH2_EINVAL, "unknown export"};
    }
    if (r * c > cap) throw Error{DH2_EINVAL, "export buffer too small"};
    *rows = (int32_t)r;
    *cols = (int32_t)c;
    if (r * c == 0) return;
    const int64_t span = (r - 1) * ld + c;
    if (is_real) {
        std::vector<double> hbuf(span);
        DH2_CHECK_CUDA(cudaMemcpyAsync(hbuf.data(), (const double*)src + off, span * sizeof(double), cudaMemcpyDeviceToHost, s));
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int64_t j = 0; j < c; ++j) {
            out[2 * j] = hbuf[j];
            out[2 * j + 1] = 0.0;
        }
    } else if (is_double) {
        std::vector<cx<double>> hbuf(span);
        DH2_CHECK_CUDA(cudaMemcpyAsync(hbuf.data(), (const cx<double>*)src + off, span * sizeof(cx<double>), cudaMemcpyDeviceToHost, s));
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < r; ++i)
            for (int64_t j = 0; j < c; ++j) {
                out[2 * (i * c + j)] = hbuf[i * ld + j].x;
                out[2 * (i * c + j) + 1] = hbuf[i * ld + j].y;
            }
    } else {
        std::vector<cx<float>> hbuf(span);
        DH2_CHECK_CUDA(cudaMemcpyAsync(hbuf.data(), (const cx<float>*)src + off, span * sizeof(cx<float>), cudaMemcpyDeviceToHost, s));
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < r; ++i)
            for (int64_t j = 0; j < c; ++j) {
                out[2 * (i * c + j)] = hbuf[i * ld + j].x;
                out[2 * (i * c + j) + 1] = hbuf[i * ld + j].y;
            }
    }
}

template <class T>
void Num<T>::export_ranks(int32_t* rr, int32_t* rc, cudaStream_t) {
    const int64_t ntc = (int64_t)hs_.aidx.size();
    for (int64_t tc = 0; tc < ntc; ++tc) {
        int32_t a = hs_.aidx[tc];
        if (rr) rr[tc] = a < 0 ? -1 : rank_[0][a];
        if (rc) rc[tc] = a < 0 ? -1 : rank_[1][a];
    }
}

std::unique_ptr<NumBase> make_numeric(const Tree& tr, Structure& st, const HostStructure& hs,
                                      const BuildParams& bp) {
    if (bp.precision == DH2_FP64) return std::unique_ptr<NumBase>(new Num<double>(tr, st, hs, bp));
    return std::unique_ptr<NumBase>(new Num<float>(tr, st, hs, bp));
}

// The Gram matrix Z^* Z of one complex FP32 matrix in FP64, as the weight factorisations
// form it (dh2_gram)
void gram_matrix(const void* z, int64_t rows, int32_t cols, int64_t ld, bool tc, void* g, cudaStream_t s) {
    DBuf<unsigned> err(1);
    DH2_CHECK_CUDA(cudaMemsetAsync(err.p, 0, sizeof(unsigned), s));
    const QRTask t{0, 0, (int32_t)rows, 0, cols, (int32_t)ld};
    EventLog ev;
    chol_qr_launch<float, float>({t}, static_cast<const cx<float>*>(z), nullptr, s, ev, err.p, tc, nullptr,
                                 static_cast<cx<double>*>(g));
    const unsigned e = read_scalar(err.p, s);
    if (e & ERR_TC_TIMEOUT) throw Error{DH2_ETIMEOUT, "dh2_gram: a bounded tensor-core wait gave up"};
    if (e) throw Error{DH2_ENUMERIC, "dh2_gram: non-finite input"};
}

}  // namespace dh2
