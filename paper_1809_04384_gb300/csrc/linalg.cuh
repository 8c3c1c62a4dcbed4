// CTA-level complex linear algebra used by the recompression kernels:
//   * cx<T>           complex scalar (T = float or double), interleaved storage
//   * cta_gemm        C = A * B with functor operands (operands may be generated
//                     on the fly, e.g. the couplings S_b), 256 threads
//   * kron_apply      X * (Ex (x) Ey (x) Ez) or X * (...)^* with the transfer
//                     matrices kept as three m x m factors
//   * tsqr_chunk      Householder update of an upper-triangular R (global) by
//                     a block of extra rows held in shared memory
//   * herm_jacobi     parallel cyclic Jacobi eigensolver for Hermitian matrices
//   * rowjac_f32      one-sided Jacobi SVD (FP32) on the rows of a complex matrix
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dh2 {

template <class T>
struct __align__(2 * sizeof(T)) cx {
    T x, y;
};

template <class T> __device__ __forceinline__ cx<T> mk(T a, T b) { return cx<T>{a, b}; }
template <class T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <class T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.x, s * a.y}; }
template <class T> __device__ __forceinline__ cx<T> conj(cx<T> a) { return {a.x, -a.y}; }
template <class T> __device__ __forceinline__ T abs2(cx<T> a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
template <class T> __device__ __forceinline__ void fma_cx(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <class T> __device__ __forceinline__ void fma_cjx(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
template <class T> __device__ __forceinline__ cx<T> zero() { return cx<T>{T(0), T(0)}; }
// smallest positive normal number
template <class T> __device__ __forceinline__ T tiny_normal();
template <> __device__ __forceinline__ float tiny_normal<float>() { return 1.17549435e-38f; }
template <> __device__ __forceinline__ double tiny_normal<double>() { return 2.2250738585072014e-308; }

template <class T>
__device__ __forceinline__ cx<T> shfl_xor(cx<T> v, int o) {
    return cx<T>{__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
}
template <class T>
__device__ __forceinline__ cx<T> warp_sum(cx<T> v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = v + shfl_xor(v, o);
    return v;
}
template <class T>
__device__ __forceinline__ T warp_sum_r(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the CTA (all threads receive the result); smem: >= 32 T
template <class T>
__device__ T block_sum(T v, T* smem) {
    v = warp_sum_r(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) smem[w] = v;
    __syncthreads();
    T r = 0;
    for (int i = 0; i < nw; ++i) r += smem[i];
    __syncthreads();
    return r;
}

// --------------------------------------------------------------------------- operands

// dense row-major complex matrix view (optionally conjugated and/or transposed)
template <class T>
struct Dense {
    const cx<T>* p;
    int64_t ld;
    bool trans, conjg;
    __device__ __forceinline__ cx<T> operator()(int i, int j) const {
        cx<T> v = trans ? p[(int64_t)j * ld + i] : p[(int64_t)i * ld + j];
        return conjg ? conj(v) : v;
    }
};

// dense view of a matrix of another precision, converted on load
template <class T, class U>
struct DenseCvt {
    const cx<U>* p;
    int64_t ld;
    bool trans, conjg;
    __device__ __forceinline__ cx<T> operator()(int i, int j) const {
        cx<U> v = trans ? p[(int64_t)j * ld + i] : p[(int64_t)i * ld + j];
        return cx<T>{T(v.x), conjg ? -T(v.y) : T(v.y)};
    }
};

// --------------------------------------------------------------------------- CTA GEMM

// C(i,j) = sum_k A(i,k) B(k,j) for 0<=i<M, 0<=j<N; `store(i, j, value)` is called
// once per output.  256 threads as 16 x 16, BM x BN output tiles, (BM/16) x (BN/16)
// outputs per thread (rows ty + 16a, columns tx + 16b), K in steps of 8.  The operands
// of the next K step are fetched (or generated) into registers while the current step
// is multiplied out of shared memory.
// One staging buffer per element type and kernel, shared by every cta_gemm call:
// 8 * (64 + 128) cx<T> = 12 KB (T=float) / 24 KB (double).
template <class T>
__device__ __forceinline__ cx<T>* gemm_smem() {
    __shared__ cx<T> buf[8 * (64 + 128)];
    return buf;
}

template <class T, int BM, int BN, class FA, class FB, class FS>
__device__ void cta_gemm_t(int M, int N, int K, const FA& A, const FB& B, const FS& store) {
    constexpr int BK = 8, TM = BM / 16, TN = BN / 16;
    constexpr int LA = BM * BK / 256, LB = BN * BK / 256;   // staged elements per thread
    static_assert(BM % 32 == 0 && BN % 32 == 0 && BM <= 64 && BN <= 128, "tile shape");
    cx<T> (*sA)[BM] = reinterpret_cast<cx<T> (*)[BM]>(gemm_smem<T>());
    cx<T> (*sB)[BN] = reinterpret_cast<cx<T> (*)[BN]>(gemm_smem<T>() + BK * BM);
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    for (int i0 = 0; i0 < M; i0 += BM) {
        for (int j0 = 0; j0 < N; j0 += BN) {
            cx<T> acc[TM][TN];
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) acc[a][b] = zero<T>();
            cx<T> ra[LA], rb[LB];
            // A is read along k (consecutive threads take consecutive k of one row),
            // B along j.
            auto fetch = [&](int k0) {
#pragma unroll
                for (int r = 0; r < LA; ++r) {
                    const int e = tid + r * 256, kk = e % BK, ii = e / BK;
                    const int gi = i0 + ii, gk = k0 + kk;
                    ra[r] = (gi < M && gk < K) ? A(gi, gk) : zero<T>();
                }
#pragma unroll
                for (int r = 0; r < LB; ++r) {
                    const int e = tid + r * 256, kk = e / BN, jj = e % BN;
                    const int gj = j0 + jj, gk = k0 + kk;
                    rb[r] = (gj < N && gk < K) ? B(gk, gj) : zero<T>();
                }
            };
            fetch(0);
            for (int k0 = 0; k0 < K; k0 += BK) {
                __syncthreads();   // the previous step's reads of sA/sB are done
#pragma unroll
                for (int r = 0; r < LA; ++r) {
                    const int e = tid + r * 256;
                    sA[e % BK][e / BK] = ra[r];
                }
#pragma unroll
                for (int r = 0; r < LB; ++r) {
                    const int e = tid + r * 256;
                    sB[e / BN][e % BN] = rb[r];
                }
                __syncthreads();
                if (k0 + BK < K) fetch(k0 + BK);
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    cx<T> av[TM], bv[TN];
#pragma unroll
                    for (int a = 0; a < TM; ++a) av[a] = sA[kk][ty + 16 * a];
#pragma unroll
                    for (int b = 0; b < TN; ++b) bv[b] = sB[kk][tx + 16 * b];
#pragma unroll
                    for (int a = 0; a < TM; ++a)
#pragma unroll
                        for (int b = 0; b < TN; ++b) fma_cx(acc[a][b], av[a], bv[b]);
                }
            }
            __syncthreads();   // sA/sB free for the next tile or the caller
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int b = 0; b < TN; ++b) {
                    const int gi = i0 + ty + 16 * a, gj = j0 + tx + 16 * b;
                    if (gi < M && gj < N) store(gi, gj, acc[a][b]);
                }
        }
    }
}

// 64 x 64 tiles: the general shape
template <class T, class FA, class FB, class FS>
__device__ void cta_gemm(int M, int N, int K, const FA& A, const FB& B, const FS& store) {
    cta_gemm_t<T, 64, 64>(M, N, K, A, B, store);
}

// Tile shape from the sizes: 32-row tiles when M <= 32 (most leaf ranks), 128-wide (FP32)
// when N > 64 (the k columns of a coupling matrix).
template <class T, class FA, class FB, class FS>
__device__ void cta_gemm_fit(int M, int N, int K, const FA& A, const FB& B, const FS& store) {
    constexpr int WIDE = sizeof(T) == 4 ? 128 : 64;   // FP64 accumulators: at most 64 wide
    if (M <= 32) {
        if (N <= 32) cta_gemm_t<T, 32, 32>(M, N, K, A, B, store);
        else if (N <= 64) cta_gemm_t<T, 32, 64>(M, N, K, A, B, store);
        else cta_gemm_t<T, 32, WIDE>(M, N, K, A, B, store);
    } else {
        if (N <= 64) cta_gemm_t<T, 64, 64>(M, N, K, A, B, store);
        else cta_gemm_t<T, 64, WIDE>(M, N, K, A, B, store);
    }
}

// --------------------------------------------------------------------------- Kronecker transfer

// out[r][nu] = sum_nu' X[r][nu'] E[nu'][nu]          (adjoint = false)
// out[r][nu'] = sum_nu X[r][nu] conj(E[nu'][nu])      (adjoint = true)
// with E[nu'][nu] = Ex[nu'x][nux] Ey[nu'y][nuy] Ez[nu'z][nuz], nu = nx + m ny + m^2 nz.
// fac: 3 consecutive m*m row-major factors (x, y, z).  `buf`: 2 * k cx<T> of shared
// memory per row in flight (rows are processed one at a time by the whole CTA).
template <class T, class FX, class FO>
__device__ void kron_apply(int rows, int m, const cx<T>* fac, bool adjoint, const FX& X,
                           const FO& out, cx<T>* buf) {
    const int k = m * m * m, mm = m * m;
    cx<T>* b0 = buf;
    cx<T>* b1 = buf + k;
    for (int r = 0; r < rows; ++r) {
        for (int v = threadIdx.x; v < k; v += blockDim.x) b0[v] = X(r, v);
        __syncthreads();
        // three passes: axis x (stride 1), y (stride m), z (stride m^2)
        for (int axis = 0; axis < 3; ++axis) {
            const cx<T>* F = fac + axis * mm;
            const int stride = axis == 0 ? 1 : (axis == 1 ? m : mm);
            cx<T>* src = (axis & 1) ? b1 : b0;
            cx<T>* dst = (axis & 1) ? b0 : b1;
            for (int v = threadIdx.x; v < k; v += blockDim.x) {
                int a = (v / stride) % m;          // output index along this axis
                int base = v - a * stride;
                cx<T> acc = zero<T>();
                for (int q = 0; q < m; ++q) {
                    cx<T> xv = src[base + q * stride];
                    // forward: sum_q X[q] F[q][a];  adjoint: sum_q X[q] conj(F[a][q])
                    cx<T> f = adjoint ? conj(F[a * m + q]) : F[q * m + a];
                    fma_cx(acc, xv, f);
                }
                dst[v] = acc;
            }
            __syncthreads();
        }
        // after three passes the result is in b1
        for (int v = threadIdx.x; v < k; v += blockDim.x) out(r, v, b1[v]);
        __syncthreads();
    }
}

// --------------------------------------------------------------------------- Householder TSQR

// R (k x k, row-major, global, upper triangular) <- R-factor of [R; W] where W is the
// block of H = 32*RPL extra rows held column-major in shared memory with leading
// dimension LDW = H + 1 (odd, so that lanes reading different columns hit different
// banks); rows >= h are zero.  Column reflectors follow LAPACK's xLARFG convention (real
// beta); the reflector of column j is e_j on the R side and its W part overwrites W[:, j].
// Blocked by NB columns: the panel is factored by warp 0 (warp-synchronous), the panel's
// reflectors are combined in compact WY form (T upper triangular, LAPACK xLARFT forward
// columnwise), and the trailing columns are updated with two small shared-memory GEMMs:
// Wm = U^H A, Wm <- T^H Wm, A <- A - U Wm.  Scratch: s_tau[NB], s_skip[NB], s_T[NB*NB],
// s_G[NB*NB], s_Wm[NB*k].
template <class T, int RPL, int NB>
__device__ void tsqr_chunk(int k, cx<T>* R, cx<T>* W, cx<T>* s_tau, int* s_skip, cx<T>* s_T,
                           cx<T>* s_G, cx<T>* s_Wm) {
    constexpr int H = 32 * RPL, LDW = H + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j0 = 0; j0 < k; j0 += NB) {
        const int nbc = min(NB, k - j0);
        // ---- panel factorisation (warp 0)
        if (warp == 0) {
            for (int jj = 0; jj < nbc; ++jj) {
                const int j = j0 + jj;
                cx<T>* wj = W + (int64_t)j * LDW;
                const cx<T> al = R[(int64_t)j * k + j];   // read before the shuffles below
                // The column is scaled by its largest entry before squaring (as LAPACK's
                // xLARFG rescales): rank-deficient columns of a merged stack hold rounding
                // remainders whose squares are denormal, and 1/|alpha - beta|^2 would overflow.
                T xmax = 0;
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    const cx<T> x = wj[lane + 32 * q];
                    xmax = fmax(xmax, fmax(fabs(x.x), fabs(x.y)));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
                if (!(xmax >= tiny_normal<T>())) {   // uniform over the warp: a numerically zero column
                    if (lane == 0) {
                        s_skip[jj] = 1;
                        s_tau[jj] = zero<T>();
                    }
                    __syncwarp();
                    continue;
                }
                const T amax = fmax(xmax, fmax(fabs(al.x), fabs(al.y)));
                const T inv = T(1) / amax;
                T xn2 = 0;
#pragma unroll
                for (int q = 0; q < RPL; ++q) xn2 += abs2(inv * wj[lane + 32 * q]);
                xn2 = warp_sum_r(xn2);
                const cx<T> als = inv * al;
                const T betas = -copysign(sqrt(abs2(als) + xn2), als.x);   // beta / amax, O(1)
                const cx<T> tauc = mk<T>((betas - als.x) / betas, als.y / betas);
                const cx<T> d = mk<T>(als.x - betas, als.y);
                const T dn = inv / abs2(d);
                const cx<T> sc = mk<T>(d.x * dn, -d.y * dn);   // 1 / (alpha - beta)
                cx<T> v[RPL];
#pragma unroll
                for (int q = 0; q < RPL; ++q) {
                    v[q] = wj[lane + 32 * q] * sc;
                    wj[lane + 32 * q] = v[q];
                }
                if (lane == 0) {
                    R[(int64_t)j * k + j] = mk<T>(betas * amax, T(0));
                    s_tau[jj] = tauc;
                    s_skip[jj] = 0;
                }
                for (int l = j + 1; l < j0 + nbc; ++l) {
                    cx<T>* wl = W + (int64_t)l * LDW;
                    const cx<T> rjl = R[(int64_t)j * k + l];
                    cx<T> s = zero<T>();
#pragma unroll
                    for (int q = 0; q < RPL; ++q) fma_cjx(s, v[q], wl[lane + 32 * q]);
                    s = warp_sum(s);
                    const cx<T> tw = tauc * (rjl + s);
#pragma unroll
                    for (int q = 0; q < RPL; ++q) wl[lane + 32 * q] = wl[lane + 32 * q] - v[q] * tw;
                    if (lane == 0) R[(int64_t)j * k + l] = rjl - tw;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        const int l0 = j0 + nbc, nl = k - l0;
        if (nl <= 0) break;
        // ---- T of the compact WY form; G[p][i] = v_p^H v_i (p < i)
        for (int pr = warp; pr < nbc * nbc; pr += nwarps) {
            const int p = pr / nbc, i = pr - p * nbc;
            if (p >= i) continue;
            const cx<T>* vp = W + (int64_t)(j0 + p) * LDW;
            const cx<T>* vi = W + (int64_t)(j0 + i) * LDW;
            cx<T> s = zero<T>();
#pragma unroll
            for (int q = 0; q < RPL; ++q) fma_cjx(s, vp[lane + 32 * q], vi[lane + 32 * q]);
            s = warp_sum(s);
            if (lane == 0) s_G[p * NB + i] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 0; i < nbc; ++i) {
                const cx<T> tau = s_skip[i] ? zero<T>() : conj(s_tau[i]);
                s_T[i * NB + i] = tau;
                for (int p = 0; p < i; ++p) {
                    cx<T> acc = zero<T>();
                    for (int q = p; q < i; ++q) fma_cx(acc, s_T[p * NB + q], s_G[q * NB + i]);
                    s_T[p * NB + i] = zero<T>() - tau * acc;
                }
            }
        }
        __syncthreads();
        // ---- Wm = U^H A over the trailing columns
        for (int idx = threadIdx.x; idx < nbc * nl; idx += blockDim.x) {
            const int p = idx / nl, l = idx - p * nl;
            const cx<T>* vp = W + (int64_t)(j0 + p) * LDW;
            const cx<T>* wl = W + (int64_t)(l0 + l) * LDW;
            cx<T> acc = R[(int64_t)(j0 + p) * k + l0 + l];
#pragma unroll 8
            for (int r = 0; r < H; ++r) fma_cjx(acc, vp[r], wl[r]);
            s_Wm[p * k + l] = acc;
        }
        __syncthreads();
        // ---- Wm <- T^H Wm and the R rows of the panel
        for (int l = threadIdx.x; l < nl; l += blockDim.x) {
            cx<T> col[NB];
#pragma unroll
            for (int p = 0; p < NB; ++p) col[p] = p < nbc ? s_Wm[p * k + l] : zero<T>();
#pragma unroll
            for (int p = NB - 1; p >= 0; --p) {
                if (p >= nbc) continue;
                cx<T> acc = zero<T>();
                for (int q = 0; q <= p; ++q) fma_cjx(acc, s_T[q * NB + p], col[q]);
                col[p] = acc;
            }
#pragma unroll
            for (int p = 0; p < NB; ++p) {
                if (p >= nbc) continue;
                s_Wm[p * k + l] = col[p];
                cx<T>* rp = R + (int64_t)(j0 + p) * k + l0 + l;
                *rp = *rp - col[p];
            }
        }
        __syncthreads();
        // ---- W <- W - U_W Wm
        for (int idx = threadIdx.x; idx < H * nl; idx += blockDim.x) {
            const int l = idx / H, r = idx - l * H;
            cx<T> acc = W[(int64_t)(l0 + l) * LDW + r];
            for (int p = 0; p < nbc; ++p) acc = acc - W[(int64_t)(j0 + p) * LDW + r] * s_Wm[p * k + l];
            W[(int64_t)(l0 + l) * LDW + r] = acc;
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------- one-sided Jacobi (FP32)

// One-sided (Hestenes) Jacobi on the rows of W (n x m, row pitch ldw, FP32 complex, global
// or shared memory): builds a unitary J (n x n) such that the rows of J^H W_in = W_out are
// mutually orthogonal, so W_in = J W_out is an SVD with the left singular vectors as the
// columns of J and the singular values as the row norms of W_out.  Jt receives J^T (row i
// of Jt is column i of J, contiguous).  Rows p, q with Gram [[a, g], [conj(g), b]],
// g = sum_j w_p[j] conj(w_q[j]) = |g| e^{i phi}, are rotated by G = diag(1, e^{-i phi}) R with
// the real Jacobi rotation R = [[c, s], [-s, c]] of [[a, |g|], [|g|, b]]:
//   zeta = (b - a) / (2|g|),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),  c = 1/sqrt(1 + t^2),
//   s = c t;  w_p <- c w_p - s e^{i phi} w_q,  w_q <- s w_p + c e^{i phi} w_q  (W <- G^H W),
//   j_p <- c j_p - s e^{-i phi} j_q,  j_q <- s j_p + c e^{-i phi} j_q  (J <- J G).
// Pairs follow the round-robin (circle) schedule, one warp per pair, a block barrier per
// round; sweeps stop when no pair has |g| > tol sqrt(a b) (pairs with |g| < 1e-30 are not
// rotated), after at most max_sweeps.  On
// return lam[i] = |w_i|^2 (FP64 sums) and order[] lists the rows by descending lam.
// Returns the number of sweeps.  All threads of the block must call it.
__device__ inline int rowjac_f32(int n, int m, cx<float>* W, int ldw, cx<float>* Jt, double* lam, int* order,
                                 int* s_flag, int max_sweeps, float tol) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        Jt[idx] = cx<float>{i == j ? 1.0f : 0.0f, 0.0f};
    }
    const int np = n + (n & 1);
    int sweep = 0;
    for (; sweep < max_sweeps && n > 1; ++sweep) {
        if (threadIdx.x == 0) *s_flag = 0;
        __syncthreads();
        for (int r = 0; r < np - 1; ++r) {
            for (int i = warp; i < np / 2; i += nwarps) {
                // circle method: position 0 fixed, the others rotate by one per round
                const int pa = i == 0 ? 0 : 1 + (i - 1 + r) % (np - 1);
                const int pb = 1 + (np - 2 - i + r) % (np - 1);
                const int p = min(pa, pb), q = max(pa, pb);
                if (q >= n) continue;   // the padding row of an odd n
                cx<float>* wp = W + (int64_t)p * ldw;
                cx<float>* wq = W + (int64_t)q * ldw;
                float a = 0.0f, b = 0.0f, gr = 0.0f, gi = 0.0f;
                for (int j = lane; j < m; j += 32) {
                    const cx<float> x = wp[j], y = wq[j];
                    a += abs2(x);
                    b += abs2(y);
                    gr += x.x * y.x + x.y * y.y;   // x conj(y)
                    gi += x.y * y.x - x.x * y.y;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    b += __shfl_xor_sync(0xffffffffu, b, o);
                    gr += __shfl_xor_sync(0xffffffffu, gr, o);
                    gi += __shfl_xor_sync(0xffffffffu, gi, o);
                }
                // |g| without underflow (rows of a tall W shrink towards zero, and the phase
                // g / |g| must keep unit modulus for the rotation to stay unitary); couplings
                // below 1e-30 are left alone
                const float ag = hypotf(gr, gi);
                if (!(ag > tol * sqrtf(a) * sqrtf(b)) || !(ag >= 1e-30f)) continue;   // warp-uniform
                if (lane == 0) *s_flag = 1;
                const float zeta = (b - a) / (2.0f * ag);
                float t;
                if (fabsf(zeta) > 1e18f) t = 0.5f / zeta;
                else t = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
                const float c = 1.0f / sqrtf(1.0f + t * t), sn = c * t;
                const cx<float> e = mk<float>(gr / ag, gi / ag);        // e^{i phi}
                const cx<float> se = mk<float>(sn * e.x, sn * e.y);     // s e^{i phi}
                const cx<float> sec = mk<float>(sn * e.x, -sn * e.y);   // s e^{-i phi}
                const cx<float> ce = mk<float>(c * e.x, c * e.y);       // c e^{i phi}
                const cx<float> cec = mk<float>(c * e.x, -c * e.y);     // c e^{-i phi}
                for (int j = lane; j < m; j += 32) {
                    const cx<float> x = wp[j], y = wq[j];
                    wp[j] = c * x - se * y;
                    wq[j] = sn * x + ce * y;
                }
                cx<float>* jp = Jt + (int64_t)p * n;
                cx<float>* jq = Jt + (int64_t)q * n;
                for (int j = lane; j < n; j += 32) {
                    const cx<float> x = jp[j], y = jq[j];
                    jp[j] = c * x - sec * y;
                    jq[j] = sn * x + cec * y;
                }
            }
            __syncthreads();
        }
        const int more = *s_flag;
        __syncthreads();
        if (!more) break;
    }
    for (int i = warp; i < n; i += nwarps) {
        double acc = 0.0;
        for (int j = lane; j < m; j += 32) acc += (double)abs2(W[(int64_t)i * ldw + j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) lam[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double li = lam[i];
        int rk = 0;
        for (int j = 0; j < n; ++j) rk += (lam[j] > li || (lam[j] == li && j < i)) ? 1 : 0;
        order[rk] = i;
    }
    __syncthreads();
    return sweep;
}

// --------------------------------------------------------------------------- Hermitian Jacobi

// Parallel cyclic Jacobi (circle schedule) for a Hermitian n x n matrix M
// (row-major, ld = n, shared or global memory).  On return the diagonal holds
// the eigenvalues and U (n x n, ld = n) the eigenvectors as columns.  rot:
// scratch of n/2+1 entries for rotation data.  Returns the number of sweeps.
template <class T>
struct JRot {
    int p, q;
    T c, s;
    cx<T> e;
};

// init_u = false: U already holds the unitary transform applied to M so far; the sweeps
// continue it (U <- U J for every rotation J)
template <class T>
__device__ int herm_jacobi(int n, cx<T>* M, cx<T>* U, JRot<T>* rot, T* red, int max_sweeps,
                           T tol, bool init_u = true) {
    const int np = n + (n & 1);
    const int half = np / 2;
    if (init_u)
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x)
            U[idx] = (idx / n == idx % n) ? mk<T>(T(1), T(0)) : zero<T>();
    __syncthreads();
    T fro = 0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) fro += abs2(M[idx]);
    fro = block_sum(fro, red);
    if (n <= 1 || fro == T(0)) return 0;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        T off = 0;
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x)
            if (idx / n != idx % n) off += abs2(M[idx]);
        off = block_sum(off, red);
        if (off <= tol * tol * fro) break;
        for (int r = 0; r < np - 1; ++r) {
            for (int pi = threadIdx.x; pi < half; pi += blockDim.x) {
                int p, q;
                if (pi == 0) {
                    p = r;
                    q = np - 1;
                } else {
                    p = (r + pi) % (np - 1);
                    q = (r - pi + np - 1) % (np - 1);
                }
                JRot<T> j;
                j.p = p;
                j.q = q;
                j.c = 1;
                j.s = 0;
                j.e = mk<T>(T(1), T(0));
                if (p < n && q < n) {
                    cx<T> apq = M[p * n + q];
                    T a = sqrt(abs2(apq));
                    if (a > T(0)) {
                        j.e = mk<T>(apq.x / a, apq.y / a);
                        T zeta = (M[q * n + q].x - M[p * n + p].x) / (T(2) * a);
                        T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                        j.c = T(1) / sqrt(T(1) + t * t);
                        j.s = t * j.c;
                    }
                }
                rot[pi] = j;
            }
            __syncthreads();
            // columns of M and U
            for (int idx = threadIdx.x; idx < half * n; idx += blockDim.x) {
                const JRot<T> j = rot[idx / n];
                const int row = idx % n;
                if (j.p >= n || j.q >= n || j.s == T(0)) continue;
                cx<T> ce = conj(j.e);
                cx<T> mp = M[row * n + j.p], mq = M[row * n + j.q];
                M[row * n + j.p] = j.c * mp - j.s * (ce * mq);
                M[row * n + j.q] = j.s * mp + j.c * (ce * mq);
                cx<T> up = U[row * n + j.p], uq = U[row * n + j.q];
                U[row * n + j.p] = j.c * up - j.s * (ce * uq);
                U[row * n + j.q] = j.s * up + j.c * (ce * uq);
            }
            __syncthreads();
            // rows of M
            for (int idx = threadIdx.x; idx < half * n; idx += blockDim.x) {
                const JRot<T> j = rot[idx / n];
                const int col = idx % n;
                if (j.p >= n || j.q >= n || j.s == T(0)) continue;
                cx<T> mp = M[j.p * n + col], mq = M[j.q * n + col];
                M[j.p * n + col] = j.c * mp - j.s * (j.e * mq);
                M[j.q * n + col] = j.s * mp + j.c * (j.e * mq);
            }
            __syncthreads();
        }
    }
    return sweep;
}

}  // namespace dh2
