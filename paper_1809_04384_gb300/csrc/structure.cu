// Cluster tree (Def. "cluster tree", Section 5 BSP), bounding boxes (Section 2),
// directions and son maps (Def. "directions", Remark "construction of
// directions"), block directions c_ts, the block tree (Def. "block tree" with
// conditions (3b),(3c)) and the (t,c) pair bookkeeping used by Section 3.2.
//
// Every floating-point value that decides an integer here is computed with
// explicit round-to-nearest intrinsics in a fixed order (and this translation
// unit is compiled with -fmad=false), so the results are bit-identical with
// any IEEE FP64 evaluation of the same expressions:
//   centroid  = ((v0 + v1) + v2) / 3
//   split     = (lo + hi) * 0.5 on the longest centroid-box axis (ties: lowest)
//   diam      = sqrt((dx*dx + dy*dy) + dz*dz) of the vertex box
//   dist      = the same norm of the per-axis gaps max(max(lo_t-hi_s, lo_s-hi_t), 0)
//   m_l       = ceil(((sqrt2 * kappa) * d_l) / eta1)
//   nearest   = argmin ((a0-b0)^2 + (a1-b1)^2) + (a2-b2)^2, ties to the lowest index
#include <mutex>

#include "structure.cuh"

namespace dh2 {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double norm3(double a, double b, double c) {
    return __dsqrt_rn(dadd(dadd(dmul(a, a), dmul(b, b)), dmul(c, c)));
}
__device__ __forceinline__ double dist2(double a0, double a1, double a2, double b0, double b1,
                                        double b2) {
    double d0 = dsub(b0, a0), d1 = dsub(b1, a1), d2 = dsub(b2, a2);
    return dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2));
}

// ------------------------------------------------------------------ block-wide helpers (256 threads)

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// exclusive scan over the block; *total receives the block sum. smem: 8 ints.
__device__ int block_excl_scan(int v, int* smem, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) smem[w] = inc;
    __syncthreads();
    if (w == 0) {
        int x = (lane < (int)(blockDim.x >> 5)) ? smem[lane] : 0;
        int y = warp_incl_scan(x);
        if (lane < (int)(blockDim.x >> 5)) smem[lane] = y - x;
        if (lane == 31) smem[8] = y;
    }
    __syncthreads();
    int r = smem[w] + inc - v;
    *total = smem[8];
    __syncthreads();
    return r;
}

__device__ double block_min(double v, double* smem) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) smem[w] = v;
    __syncthreads();
    double r = smem[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fmin(r, smem[i]);
    __syncthreads();
    return r;
}

__device__ double block_max(double v, double* smem) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) smem[w] = v;
    __syncthreads();
    double r = smem[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fmax(r, smem[i]);
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ geometry per element

__global__ void k_geom(const double* __restrict__ vert, const int32_t* __restrict__ tri, int64_t n,
                       bool point_mode, double* cent, double* tlo, double* thi) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a, b, c;
    if (point_mode) {
        a = b = c = (int32_t)i;
    } else {
        a = tri[3 * i];
        b = tri[3 * i + 1];
        c = tri[3 * i + 2];
    }
    for (int ax = 0; ax < 3; ++ax) {
        double v0 = vert[3 * a + ax], v1 = vert[3 * b + ax], v2 = vert[3 * c + ax];
        cent[ax * n + i] = ddiv(dadd(dadd(v0, v1), v2), 3.0);
        tlo[ax * n + i] = fmin(fmin(v0, v1), v2);
        thi[ax * n + i] = fmax(fmax(v0, v1), v2);
    }
}

// ------------------------------------------------------------------ BSP, one level at a time

// One CTA per cluster of the level: vertex box; for clusters above leaf_max
// the split axis/value and the size of the left son.  mode[t]: 0 = leaf,
// 1 = split by value, 2 = median split.
__global__ void k_level_boxes(int32_t lv_begin, const int32_t* __restrict__ offset,
                              const int32_t* __restrict__ size, const int32_t* __restrict__ perm,
                              const double* __restrict__ cent, const double* __restrict__ tlo,
                              const double* __restrict__ thi, int64_t n, int32_t leaf_max,
                              int32_t nc_cap, double* lo, double* hi, int8_t* mode,
                              int8_t* axis_out, double* split_out, int32_t* nleft) {
    __shared__ double sm[32];
    __shared__ int smi[16];
    const int32_t t = lv_begin + blockIdx.x;
    const int32_t off = offset[t], sz = size[t];
    for (int ax = 0; ax < 3; ++ax) {
        double mn = INFINITY, mx = -INFINITY;
        for (int32_t i = threadIdx.x; i < sz; i += blockDim.x) {
            int32_t e = perm[off + i];
            mn = fmin(mn, tlo[ax * n + e]);
            mx = fmax(mx, thi[ax * n + e]);
        }
        mn = block_min(mn, sm);
        mx = block_max(mx, sm);
        if (threadIdx.x == 0) {
            lo[ax * nc_cap + t] = mn;
            hi[ax * nc_cap + t] = mx;
        }
    }
    if (sz <= leaf_max) {
        if (threadIdx.x == 0) mode[t] = 0;
        return;
    }
    double clo[3], chi[3];
    for (int ax = 0; ax < 3; ++ax) {
        double mn = INFINITY, mx = -INFINITY;
        for (int32_t i = threadIdx.x; i < sz; i += blockDim.x) {
            double c = cent[ax * n + perm[off + i]];
            mn = fmin(mn, c);
            mx = fmax(mx, c);
        }
        clo[ax] = block_min(mn, sm);
        chi[ax] = block_max(mx, sm);
    }
    int axis = 0;
    double ext0 = dsub(chi[0], clo[0]), ext1 = dsub(chi[1], clo[1]), ext2 = dsub(chi[2], clo[2]);
    double best = ext0;
    if (ext1 > best) { axis = 1; best = ext1; }
    if (ext2 > best) { axis = 2; best = ext2; }
    const double split = dmul(dadd(clo[axis], chi[axis]), 0.5);
    int cnt = 0;
    for (int32_t i = threadIdx.x; i < sz; i += blockDim.x)
        cnt += cent[axis * n + perm[off + i]] < split ? 1 : 0;
    int total;
    block_excl_scan(cnt, smi, &total);
    if (threadIdx.x == 0) {
        axis_out[t] = (int8_t)axis;
        split_out[t] = split;
        if (total == 0 || total == sz) {
            mode[t] = 2;
            nleft[t] = sz / 2;
        } else {
            mode[t] = 1;
            nleft[t] = total;
        }
    }
}

// Single CTA: numbers the sons of the level's split clusters (breadth first,
// left son first) and writes their records.  *next_count = sons created.
__global__ void k_level_sons(int32_t lv_begin, int32_t lv_count, const int8_t* __restrict__ mode,
                             const int32_t* __restrict__ nleft, int32_t* offset, int32_t* size,
                             int32_t* parent, int32_t* son0, int32_t* son1, int32_t* level,
                             int32_t lvl, int32_t* next_count) {
    __shared__ int smi[16];
    const int32_t base_next = lv_begin + lv_count;
    int running = 0;
    for (int32_t c0 = 0; c0 < lv_count; c0 += blockDim.x) {
        int32_t i = c0 + threadIdx.x;
        int32_t t = lv_begin + i;
        int f = (i < lv_count && mode[t] != 0) ? 1 : 0;
        int total;
        int r = block_excl_scan(f, smi, &total) + running;
        if (i < lv_count) {
            if (f) {
                int32_t a = base_next + 2 * r, b = a + 1;
                son0[t] = a;
                son1[t] = b;
                int32_t nl = nleft[t];
                offset[a] = offset[t];
                size[a] = nl;
                offset[b] = offset[t] + nl;
                size[b] = size[t] - nl;
                parent[a] = t;
                parent[b] = t;
                level[a] = lvl + 1;
                level[b] = lvl + 1;
                son0[a] = son1[a] = son0[b] = son1[b] = -1;
            } else {
                son0[t] = -1;
                son1[t] = -1;
            }
        }
        running += total;
    }
    if (threadIdx.x == 0) *next_count = 2 * running;
}

// One CTA per cluster of the level (leaves return): stable partition of the
// cluster's segment of perm into left / right son.
__global__ void k_level_partition(int32_t lv_begin, const int32_t* __restrict__ offset,
                                  const int32_t* __restrict__ size, const int8_t* __restrict__ mode,
                                  const int8_t* __restrict__ axis_in,
                                  const double* __restrict__ split_in,
                                  const int32_t* __restrict__ nleft, const double* __restrict__ cent,
                                  int64_t n, int32_t* perm, int32_t* tmp) {
    __shared__ int smi[16];
    const int32_t t = lv_begin + blockIdx.x;
    const int md = mode[t];
    if (md == 0) return;
    const int32_t off = offset[t], sz = size[t], nl = nleft[t];
    const int axis = axis_in[t];
    const double split = split_in[t];
    const double* key = cent + axis * n;
    int run_l = 0, run_r = 0;
    for (int32_t c0 = 0; c0 < sz; c0 += blockDim.x) {
        int32_t i = c0 + threadIdx.x;
        int f = 0;
        int32_t e = 0;
        if (i < sz) {
            e = perm[off + i];
            double ke = key[e];
            if (md == 1) {
                f = ke < split;
            } else {
                // rank of (key, element index) among the segment
                int32_t rank = 0;
                for (int32_t j = 0; j < sz; ++j) {
                    int32_t g = perm[off + j];
                    double kg = key[g];
                    rank += (kg < ke || (kg == ke && g < e)) ? 1 : 0;
                }
                f = rank < nl;
            }
        }
        int tot_l;
        int pl = block_excl_scan(f, smi, &tot_l);
        if (i < sz) {
            if (f)
                tmp[off + run_l + pl] = e;
            else
                tmp[off + nl + run_r + (i - c0 - pl)] = e;
        }
        int cnt_chunk = min((int32_t)blockDim.x, sz - c0);
        run_l += tot_l;
        run_r += cnt_chunk - tot_l;
    }
    __syncthreads();
    for (int32_t i = threadIdx.x; i < sz; i += blockDim.x) perm[off + i] = tmp[off + i];
}

__global__ void k_iota(int32_t* p, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}

__global__ void k_root(int32_t* offset, int32_t* size, int32_t* parent, int32_t* level, int32_t n) {
    offset[0] = 0;
    size[0] = n;
    parent[0] = -1;
    level[0] = 0;
}

// ------------------------------------------------------------------ quadrature nodes (floating only)

__constant__ double c_bary3[3][3];
__constant__ double c_bary7[7][3];

__global__ void k_quadrature(const double* __restrict__ vert, const int32_t* __restrict__ tri,
                             int64_t n, bool point_mode, double* area, double* x3, double* x7) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t id[3];
    if (point_mode) {
        id[0] = id[1] = id[2] = (int32_t)i;
    } else {
        for (int j = 0; j < 3; ++j) id[j] = tri[3 * i + j];
    }
    double v[3][3];
    for (int j = 0; j < 3; ++j)
        for (int a = 0; a < 3; ++a) v[j][a] = vert[3 * id[j] + a];
    double e1[3], e2[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = v[1][a] - v[0][a];
        e2[a] = v[2][a] - v[0][a];
    }
    double cx = e1[1] * e2[2] - e1[2] * e2[1];
    double cy = e1[2] * e2[0] - e1[0] * e2[2];
    double cz = e1[0] * e2[1] - e1[1] * e2[0];
    area[i] = point_mode ? 1.0 : 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    for (int q = 0; q < 3; ++q)
        for (int a = 0; a < 3; ++a)
            x3[(i * 3 + q) * 3 + a] =
                (c_bary3[q][0] * v[0][a] + c_bary3[q][1] * v[1][a]) + c_bary3[q][2] * v[2][a];
    for (int q = 0; q < 7; ++q)
        for (int a = 0; a < 3; ++a)
            x7[(i * 7 + q) * 3 + a] =
                (c_bary7[q][0] * v[0][a] + c_bary7[q][1] * v[1][a]) + c_bary7[q][2] * v[2][a];
}

// ------------------------------------------------------------------ cluster geometry

__global__ void k_diam(const double* __restrict__ lo, const double* __restrict__ hi, int32_t nc,
                       int32_t cap, double* diam) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc) return;
    diam[t] = norm3(dsub(hi[t], lo[t]), dsub(hi[cap + t], lo[cap + t]),
                    dsub(hi[2 * cap + t], lo[2 * cap + t]));
}

// ------------------------------------------------------------------ directions

__global__ void k_msplit(const double* __restrict__ dmax, int32_t nlev, double kappa, double eta1,
                         int32_t* msplit) {
    int32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlev) return;
    double d = dmax[l];
    if (dmul(kappa, d) <= eta1) {
        msplit[l] = 0;
    } else {
        const double sqrt2 = 1.4142135623730951;
        msplit[l] = (int32_t)ceil(ddiv(dmul(dmul(sqrt2, kappa), d), eta1));
    }
}

// face-centre directions of level l (faces +x,-x,+y,-y,+z,-z; first free axis outer)
__global__ void k_dirs(int32_t m, int32_t count, double* out) {
    int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= count) return;
    if (m == 0) {
        out[3 * g] = out[3 * g + 1] = out[3 * g + 2] = 0.0;
        return;
    }
    int32_t face = g / (m * m), r = g % (m * m);
    int32_t i = r / m, j = r % m;
    int32_t axis = face >> 1;
    double sign = (face & 1) ? -1.0 : 1.0;
    int32_t b = axis == 0 ? 1 : 0;
    int32_t c = axis == 2 ? 1 : 2;
    double v[3];
    v[axis] = sign;
    v[b] = dadd(-1.0, ddiv((double)(2 * i + 1), (double)m));
    v[c] = dadd(-1.0, ddiv((double)(2 * j + 1), (double)m));
    double nrm = norm3(v[0], v[1], v[2]);
    out[3 * g] = ddiv(v[0], nrm);
    out[3 * g + 1] = ddiv(v[1], nrm);
    out[3 * g + 2] = ddiv(v[2], nrm);
}

// sd_l: nearest direction of level l+1 (ties to the lowest index)
__global__ void k_sd(const double* __restrict__ d0, int32_t n0, const double* __restrict__ d1,
                     int32_t n1, int32_t* sd) {
    int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n0) return;
    double a0 = d0[3 * g], a1 = d0[3 * g + 1], a2 = d0[3 * g + 2];
    int32_t best = 0;
    double bd = dist2(a0, a1, a2, d1[0], d1[1], d1[2]);
    for (int32_t j = 1; j < n1; ++j) {
        double dd = dist2(a0, a1, a2, d1[3 * j], d1[3 * j + 1], d1[3 * j + 2]);
        if (dd < bd) {
            bd = dd;
            best = j;
        }
    }
    sd[g] = best;
}

// ------------------------------------------------------------------ block tree

struct ClusterGeom {
    const double* lo;
    const double* hi;
    const double* diam;
    int32_t cap;
};

__device__ __forceinline__ bool is_admissible(const ClusterGeom& g, int32_t t, int32_t s,
                                              double kappa, double eta2) {
    double gap[3];
    for (int a = 0; a < 3; ++a) {
        double x = dsub(g.lo[a * g.cap + t], g.hi[a * g.cap + s]);
        double y = dsub(g.lo[a * g.cap + s], g.hi[a * g.cap + t]);
        gap[a] = fmax(fmax(x, y), 0.0);
    }
    double dist = norm3(gap[0], gap[1], gap[2]);
    double dt = g.diam[t], ds = g.diam[s];
    double dmx = fmax(dt, ds);
    double d2 = fmax(dmul(dt, dt), dmul(ds, ds));
    double ed = dmul(eta2, dist);
    return dmx <= ed && dmul(kappa, d2) <= ed;
}

// c_ts: best approximation of (m_t - m_s)/|m_t - m_s| in D_l
__device__ int32_t block_direction(const ClusterGeom& g, int32_t t, int32_t s,
                                   const double* __restrict__ dirs, int32_t nd) {
    if (nd == 1) return 0;
    double d[3];
    for (int a = 0; a < 3; ++a) {
        double mt = dmul(dadd(g.lo[a * g.cap + t], g.hi[a * g.cap + t]), 0.5);
        double ms = dmul(dadd(g.lo[a * g.cap + s], g.hi[a * g.cap + s]), 0.5);
        d[a] = dsub(mt, ms);
    }
    double nrm = norm3(d[0], d[1], d[2]);
    if (nrm == 0.0) return 0;
    double u0 = ddiv(d[0], nrm), u1 = ddiv(d[1], nrm), u2 = ddiv(d[2], nrm);
    int32_t best = 0;
    double bd = dist2(u0, u1, u2, dirs[0], dirs[1], dirs[2]);
    for (int32_t j = 1; j < nd; ++j) {
        double dd = dist2(u0, u1, u2, dirs[3 * j], dirs[3 * j + 1], dirs[3 * j + 2]);
        if (dd < bd) {
            bd = dd;
            best = j;
        }
    }
    return best;
}

// type: 0 admissible, 1 subdivide, 2 nearfield; f_adm / f_sub / f_near flags for the scans
__global__ void k_classify(const int32_t* __restrict__ ft, const int32_t* __restrict__ fs, int64_t np,
                           ClusterGeom g, const int32_t* __restrict__ son0, double kappa, double eta2,
                           const double* __restrict__ dirs_l, int32_t nd, int32_t* f_adm,
                           int32_t* f_sub, int32_t* f_near, int32_t* cdir) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    int32_t t = ft[p], s = fs[p];
    int a = 0, sub = 0, nr = 0;
    int32_t c = 0;
    if (is_admissible(g, t, s, kappa, eta2)) {
        a = 1;
        c = block_direction(g, t, s, dirs_l, nd);
    } else if (son0[t] >= 0 && son0[s] >= 0) {
        sub = 4;
    } else {
        nr = 1;
    }
    f_adm[p] = a;
    f_sub[p] = sub;
    f_near[p] = nr;
    cdir[p] = c;
}

__global__ void k_emit(const int32_t* __restrict__ ft, const int32_t* __restrict__ fs, int64_t np,
                       const int32_t* __restrict__ f_adm, const int32_t* __restrict__ o_adm,
                       const int32_t* __restrict__ f_sub, const int32_t* __restrict__ o_sub,
                       const int32_t* __restrict__ f_near, const int32_t* __restrict__ o_near,
                       const int32_t* __restrict__ cdir, const int32_t* __restrict__ son0,
                       const int32_t* __restrict__ son1, int64_t adm_base, int32_t* adm_t,
                       int32_t* adm_s, int32_t* adm_c, int64_t near_base, int32_t* near_t,
                       int32_t* near_s, int32_t* nt, int32_t* ns) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    int32_t t = ft[p], s = fs[p];
    if (f_adm[p]) {
        int64_t q = adm_base + o_adm[p];
        adm_t[q] = t;
        adm_s[q] = s;
        adm_c[q] = cdir[p];
    } else if (f_sub[p]) {
        int64_t q = o_sub[p];
        int32_t t0 = son0[t], t1 = son1[t], s0 = son0[s], s1 = son1[s];
        nt[q] = t0; ns[q] = s0;
        nt[q + 1] = t0; ns[q + 1] = s1;
        nt[q + 2] = t1; ns[q + 2] = s0;
        nt[q + 3] = t1; ns[q + 3] = s1;
    } else if (f_near[p]) {
        int64_t q = near_base + o_near[p];
        near_t[q] = t;
        near_s[q] = s;
    }
}

// ------------------------------------------------------------------ pairs

__global__ void k_ndir_per_cluster(const int32_t* __restrict__ level, int32_t nc,
                                   const int32_t* __restrict__ ndir_l, int32_t* cnt) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nc) cnt[t] = ndir_l[level[t]];
}

__global__ void k_tc_cluster(const int32_t* __restrict__ tc_base, const int32_t* __restrict__ level,
                             const int32_t* __restrict__ ndir_l, int32_t nc, int32_t* tc_cluster) {
    int32_t t = blockIdx.x;
    if (t >= nc) return;
    int32_t b = tc_base[t], nd = ndir_l[level[t]];
    for (int32_t c = threadIdx.x; c < nd; c += blockDim.x) tc_cluster[b + c] = t;
}

__global__ void k_block_keys(const int32_t* __restrict__ bt, const int32_t* __restrict__ bs,
                             const int32_t* __restrict__ bc, int64_t nb,
                             const int32_t* __restrict__ tc_base, int32_t* rkey, int32_t* ckey,
                             int32_t* ids) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nb) return;
    rkey[b] = tc_base[bt[b]] + bc[b];
    ckey[b] = tc_base[bs[b]] + bc[b];
    ids[b] = (int32_t)b;
}

__global__ void k_histogram(const int32_t* __restrict__ keys, int64_t n, int32_t* cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[keys[i]], 1);
}

__global__ void k_active_seed(const int32_t* __restrict__ rcnt, const int32_t* __restrict__ ccnt,
                              int64_t ntc, int8_t* active) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < ntc) active[i] = (rcnt[i] + ccnt[i]) > 0;
}

// closes the active set downward for the pairs of one level
__global__ void k_active_close(int32_t tc_begin, int32_t tc_end, const int32_t* __restrict__ tc_cluster,
                               const int32_t* __restrict__ tc_base, const int32_t* __restrict__ son0,
                               const int32_t* __restrict__ son1, const int32_t* __restrict__ sd_l,
                               int8_t* active) {
    int32_t tc = tc_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (tc >= tc_end || !active[tc]) return;
    int32_t t = tc_cluster[tc];
    if (son0[t] < 0) return;
    int32_t c1 = sd_l[tc - tc_base[t]];
    active[tc_base[son0[t]] + c1] = 1;
    active[tc_base[son1[t]] + c1] = 1;
}

__global__ void k_to_i32(const int8_t* __restrict__ a, int64_t n, int32_t* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i];
}

__global__ void k_active_lists(const int8_t* __restrict__ active, const int32_t* __restrict__ pos,
                               int64_t ntc, const int32_t* __restrict__ tc_cluster,
                               const int32_t* __restrict__ tc_base, int32_t* aidx, int32_t* alist,
                               int32_t* a_t, int32_t* a_c) {
    int64_t tc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tc >= ntc) return;
    if (active[tc]) {
        int32_t a = pos[tc];
        aidx[tc] = a;
        alist[a] = (int32_t)tc;
        int32_t t = tc_cluster[tc];
        a_t[a] = t;
        a_c[a] = (int32_t)tc - tc_base[t];
    } else {
        aidx[tc] = -1;
    }
}

__global__ void k_isd_keys(const int32_t* __restrict__ sd, int32_t begin, int32_t count,
                           int32_t next_off, int32_t* keys, int32_t* vals) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    keys[begin + i] = next_off + sd[begin + i];
    vals[begin + i] = begin + i;
}

int bits_for(int64_t n) {
    int b = 1;
    while ((int64_t(1) << b) <= n) ++b;
    return b;
}

}  // namespace

// ============================================================================ host: tree

void build_tree_gpu(Tree& tr, cudaStream_t s) {
    const int64_t n = tr.n;
    const int32_t cap = (int32_t)(2 * n + 1);
    tr.cent.alloc(3 * n);
    tr.tlo.alloc(3 * n);
    tr.thi.alloc(3 * n);
    k_geom<<<grid_for(n, kThreads), kThreads, 0, s>>>(tr.vert.p, tr.tri.p, n, tr.point_mode,
                                                      tr.cent.p, tr.tlo.p, tr.thi.p);
    DH2_CHECK_LAUNCH("k_geom");
    tr.perm.alloc(n);
    DBuf<int32_t> tmp(n);
    k_iota<<<grid_for(n, kThreads), kThreads, 0, s>>>(tr.perm.p, n);
    DH2_CHECK_LAUNCH("k_iota");
    DBuf<int32_t> offset(cap), size(cap), parent(cap), son0(cap), son1(cap), level(cap);
    DBuf<double> lo(3 * (size_t)cap), hi(3 * (size_t)cap), split(cap);
    DBuf<int8_t> mode(cap), axis(cap);
    DBuf<int32_t> nleft(cap), next_count(1);
    k_root<<<1, 1, 0, s>>>(offset.p, size.p, parent.p, level.p, (int32_t)n);
    DH2_CHECK_LAUNCH("k_root");

    std::vector<int32_t> lstart{0};
    int32_t lv_begin = 0, lv_count = 1, lvl = 0;
    while (lv_count > 0) {
        k_level_boxes<<<lv_count, kThreads, 0, s>>>(lv_begin, offset.p, size.p, tr.perm.p, tr.cent.p,
                                                    tr.tlo.p, tr.thi.p, n, tr.leaf_max, cap, lo.p,
                                                    hi.p, mode.p, axis.p, split.p, nleft.p);
        DH2_CHECK_LAUNCH("k_level_boxes");
        k_level_sons<<<1, kThreads, 0, s>>>(lv_begin, lv_count, mode.p, nleft.p, offset.p, size.p,
                                            parent.p, son0.p, son1.p, level.p, lvl, next_count.p);
        DH2_CHECK_LAUNCH("k_level_sons");
        k_level_partition<<<lv_count, kThreads, 0, s>>>(lv_begin, offset.p, size.p, mode.p, axis.p,
                                                        split.p, nleft.p, tr.cent.p, n, tr.perm.p,
                                                        tmp.p);
        DH2_CHECK_LAUNCH("k_level_partition");
        int32_t nxt = read_scalar(next_count.p, s);
        lv_begin += lv_count;
        lstart.push_back(lv_begin);
        lv_count = nxt;
        ++lvl;
    }
    tr.nc = lv_begin;
    tr.depth = (int32_t)lstart.size() - 2;
    tr.level_start = lstart;
    // compact the cluster arrays to nc entries
    const int32_t nc = tr.nc;
    auto shrink = [&](DBuf<int32_t>& src, DBuf<int32_t>& dst) {
        dst.alloc(nc);
        DH2_CHECK_CUDA(cudaMemcpyAsync(dst.p, src.p, nc * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    };
    shrink(offset, tr.offset);
    shrink(size, tr.size);
    shrink(parent, tr.parent);
    shrink(son0, tr.son0);
    shrink(son1, tr.son1);
    shrink(level, tr.level);
    tr.lo.alloc(3 * (size_t)nc);
    tr.hi.alloc(3 * (size_t)nc);
    for (int a = 0; a < 3; ++a) {
        DH2_CHECK_CUDA(cudaMemcpyAsync(tr.lo.p + a * nc, lo.p + (size_t)a * cap, nc * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
        DH2_CHECK_CUDA(cudaMemcpyAsync(tr.hi.p + a * nc, hi.p + (size_t)a * cap, nc * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
    }
    DH2_CHECK_CUDA(cudaStreamSynchronize(s));
}

void prepare_quadrature(Tree& tr, cudaStream_t s) {
    // the rules' barycentric coordinates go to constant memory once per device
    static std::mutex mu;
    static bool ready[64] = {};
    int dev = 0;
    DH2_CHECK_CUDA(cudaGetDevice(&dev));
    DH2_REQUIRE(dev < 64, "prepare_quadrature: device ordinal >= 64");
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[dev]) {
        const double b3[3][3] = {{2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0},
                                 {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0},
                                 {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0}};
        const double s15 = sqrt(15.0);
        const double a1 = (6.0 - s15) / 21.0, b1 = (9.0 + 2.0 * s15) / 21.0;
        const double a2 = (6.0 + s15) / 21.0, b2 = (9.0 - 2.0 * s15) / 21.0;
        const double b7[7][3] = {{1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0}, {b1, a1, a1}, {a1, b1, a1},
                                 {a1, a1, b1}, {b2, a2, a2}, {a2, b2, a2}, {a2, a2, b2}};
        DH2_CHECK_CUDA(cudaMemcpyToSymbol(c_bary3, b3, sizeof(b3)));
        DH2_CHECK_CUDA(cudaMemcpyToSymbol(c_bary7, b7, sizeof(b7)));
        ready[dev] = true;
    }
    const int64_t n = tr.n;
    tr.area.alloc(n);
    tr.x3.alloc(9 * n);
    tr.x7.alloc(21 * n);
    k_quadrature<<<grid_for(n, kThreads), kThreads, 0, s>>>(tr.vert.p, tr.tri.p, n, tr.point_mode,
                                                            tr.area.p, tr.x3.p, tr.x7.p);
    DH2_CHECK_LAUNCH("k_quadrature");
}

// ============================================================================ host: structure

void build_structure(const Tree& tr, Structure& st, double kappa, double eta1, double eta2,
                     cudaStream_t s) {
    st.kappa = kappa;
    st.eta1 = eta1;
    st.eta2 = eta2;
    st.depth = tr.depth;
    st.nc = tr.nc;
    const int32_t nc = tr.nc, nlev = tr.depth + 1;
    ClusterGeom g{tr.lo.p, tr.hi.p, nullptr, nc};

    // --- diameters and d_l
    st.diam.alloc(nc);
    k_diam<<<grid_for(nc, kThreads), kThreads, 0, s>>>(tr.lo.p, tr.hi.p, nc, nc, st.diam.p);
    DH2_CHECK_LAUNCH("k_diam");
    g.diam = st.diam.p;
    st.dmax.resize(nlev);
    for (int l = 0; l < nlev; ++l)
        st.dmax[l] = reduce_max_f64(st.diam.p + tr.level_start[l],
                                    tr.level_start[l + 1] - tr.level_start[l], s);
    DBuf<double> dmax_d(nlev);
    dmax_d.upload(st.dmax.data(), nlev, s);
    DBuf<int32_t> msplit_d(nlev);
    k_msplit<<<1, 64, 0, s>>>(dmax_d.p, nlev, kappa, eta1, msplit_d.p);
    DH2_CHECK_LAUNCH("k_msplit");
    st.msplit = msplit_d.to_host(s);
    st.ndir.resize(nlev);
    st.dir_off.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
        int64_t m = st.msplit[l];
        if (m > 0 && 6 * m * m > (int64_t(1) << 24))
            throw Error{DH2_EUNSUPPORTED, "too many directions on one level"};
        st.ndir[l] = m == 0 ? 1 : (int32_t)(6 * m * m);
        st.dir_off[l + 1] = st.dir_off[l] + st.ndir[l];
    }
    const int32_t ndtot = st.dir_off[nlev];
    st.dirs.alloc(3 * (size_t)ndtot);
    st.sd.alloc(ndtot);
    st.sd.zero(s);
    for (int l = 0; l < nlev; ++l) {
        k_dirs<<<grid_for(st.ndir[l], kThreads), kThreads, 0, s>>>(st.msplit[l], st.ndir[l],
                                                                   st.dirs.p + 3 * st.dir_off[l]);
        DH2_CHECK_LAUNCH("k_dirs");
    }
    for (int l = 0; l + 1 < nlev; ++l) {
        k_sd<<<grid_for(st.ndir[l], kThreads), kThreads, 0, s>>>(
            st.dirs.p + 3 * st.dir_off[l], st.ndir[l], st.dirs.p + 3 * st.dir_off[l + 1],
            st.ndir[l + 1], st.sd.p + st.dir_off[l]);
        DH2_CHECK_LAUNCH("k_sd");
    }
    st.dir_off_d.alloc(nlev + 1);
    st.dir_off_d.upload(st.dir_off.data(), nlev + 1, s);
    st.ndir_d.alloc(nlev);
    st.ndir_d.upload(st.ndir.data(), nlev, s);

    // --- sd^{-1} as CSR over global directions (parents sorted ascending)
    {
        DBuf<int32_t> keys(ndtot), vals(ndtot), ks(ndtot);
        st.isd_idx.alloc(ndtot);
        int32_t nkeys = 0;
        for (int l = 0; l + 1 < nlev; ++l) {
            k_isd_keys<<<grid_for(st.ndir[l], kThreads), kThreads, 0, s>>>(
                st.sd.p, st.dir_off[l], st.ndir[l], st.dir_off[l + 1], keys.p, vals.p);
            DH2_CHECK_LAUNCH("k_isd_keys");
            nkeys += st.ndir[l];
        }
        DBuf<int32_t> cnt(ndtot + 1);
        cnt.zero(s);
        st.isd_ptr.alloc(ndtot + 1);
        if (nkeys > 0) {
            sort_pairs_i32(keys.p, ks.p, vals.p, st.isd_idx.p, nkeys, bits_for(ndtot), s);
            k_histogram<<<grid_for(nkeys, kThreads), kThreads, 0, s>>>(ks.p, nkeys, cnt.p);
            DH2_CHECK_LAUNCH("k_histogram");
        }
        exclusive_scan_i32(cnt.p, st.isd_ptr.p, ndtot + 1, s);
    }

    // --- block tree, breadth first
    {
        DBuf<int32_t> ft(1), fs(1);
        int32_t zero = 0;
        ft.upload(&zero, 1, s);
        fs.upload(&zero, 1, s);
        int64_t np = 1;
        std::vector<std::pair<DBuf<int32_t>, DBuf<int32_t>>> adm_parts, near_parts;
        std::vector<DBuf<int32_t>> admc_parts;
        std::vector<int64_t> adm_sizes, near_sizes;
        int lvl = 0;
        while (np > 0) {
            DBuf<int32_t> fa(np), fsub(np), fn(np), oa(np), osub(np), on(np), cd(np);
            k_classify<<<grid_for(np, kThreads), kThreads, 0, s>>>(
                ft.p, fs.p, np, g, tr.son0.p, kappa, eta2, st.dirs.p + 3 * st.dir_off[lvl],
                st.ndir[lvl], fa.p, fsub.p, fn.p, cd.p);
            DH2_CHECK_LAUNCH("k_classify");
            int64_t na = exclusive_scan_i32(fa.p, oa.p, np, s);
            int64_t nsub = exclusive_scan_i32(fsub.p, osub.p, np, s);
            int64_t nn = exclusive_scan_i32(fn.p, on.p, np, s);
            DBuf<int32_t> at(na), as(na), ac(na), nt_(nn), ns_(nn), nft(nsub), nfs(nsub);
            k_emit<<<grid_for(np, kThreads), kThreads, 0, s>>>(
                ft.p, fs.p, np, fa.p, oa.p, fsub.p, osub.p, fn.p, on.p, cd.p, tr.son0.p, tr.son1.p,
                0, at.p, as.p, ac.p, 0, nt_.p, ns_.p, nft.p, nfs.p);
            DH2_CHECK_LAUNCH("k_emit");
            adm_parts.emplace_back(std::move(at), std::move(as));
            admc_parts.push_back(std::move(ac));
            near_parts.emplace_back(std::move(nt_), std::move(ns_));
            adm_sizes.push_back(na);
            near_sizes.push_back(nn);
            ft = std::move(nft);
            fs = std::move(nfs);
            np = nsub;
            ++lvl;
            if (lvl > tr.depth && np > 0) throw Error{DH2_ECUDA, "block tree deeper than cluster tree"};
        }
        int64_t na = 0, nn = 0;
        for (auto x : adm_sizes) na += x;
        for (auto x : near_sizes) nn += x;
        st.nadm = na;
        st.nnear = nn;
        st.adm_t.alloc(na);
        st.adm_s.alloc(na);
        st.adm_c.alloc(na);
        st.near_t.alloc(nn);
        st.near_s.alloc(nn);
        int64_t oa = 0, on = 0;
        for (size_t i = 0; i < adm_sizes.size(); ++i) {
            size_t b = adm_sizes[i] * sizeof(int32_t);
            if (b) {
                DH2_CHECK_CUDA(cudaMemcpyAsync(st.adm_t.p + oa, adm_parts[i].first.p, b, cudaMemcpyDeviceToDevice, s));
                DH2_CHECK_CUDA(cudaMemcpyAsync(st.adm_s.p + oa, adm_parts[i].second.p, b, cudaMemcpyDeviceToDevice, s));
                DH2_CHECK_CUDA(cudaMemcpyAsync(st.adm_c.p + oa, admc_parts[i].p, b, cudaMemcpyDeviceToDevice, s));
            }
            oa += adm_sizes[i];
            b = near_sizes[i] * sizeof(int32_t);
            if (b) {
                DH2_CHECK_CUDA(cudaMemcpyAsync(st.near_t.p + on, near_parts[i].first.p, b, cudaMemcpyDeviceToDevice, s));
                DH2_CHECK_CUDA(cudaMemcpyAsync(st.near_s.p + on, near_parts[i].second.p, b, cudaMemcpyDeviceToDevice, s));
            }
            on += near_sizes[i];
        }
        DH2_CHECK_CUDA(cudaStreamSynchronize(s));
    }

    // --- pairs (t,c)
    {
        DBuf<int32_t> cnt(nc);
        k_ndir_per_cluster<<<grid_for(nc, kThreads), kThreads, 0, s>>>(tr.level.p, nc, st.ndir_d.p, cnt.p);
        DH2_CHECK_LAUNCH("k_ndir_per_cluster");
        st.tc_base.alloc(nc);
        st.ntc = exclusive_scan_i32(cnt.p, st.tc_base.p, nc, s);
        if (st.ntc >= (int64_t(1) << 30)) throw Error{DH2_EUNSUPPORTED, "too many (t,c) pairs"};
        st.tc_cluster.alloc(st.ntc);
        k_tc_cluster<<<nc, 128, 0, s>>>(st.tc_base.p, tr.level.p, st.ndir_d.p, nc, st.tc_cluster.p);
        DH2_CHECK_LAUNCH("k_tc_cluster");
    }
    const int64_t ntc = st.ntc, na = st.nadm;
    {
        DBuf<int32_t> rkey(na), ckey(na), ids(na), ks(na), rcnt(ntc + 1), ccnt(ntc + 1);
        rcnt.zero(s);
        ccnt.zero(s);
        st.row_idx.alloc(na);
        st.col_idx.alloc(na);
        st.row_ptr.alloc(ntc + 1);
        st.col_ptr.alloc(ntc + 1);
        if (na > 0) {
            k_block_keys<<<grid_for(na, kThreads), kThreads, 0, s>>>(st.adm_t.p, st.adm_s.p, st.adm_c.p,
                                                                     na, st.tc_base.p, rkey.p, ckey.p, ids.p);
            DH2_CHECK_LAUNCH("k_block_keys");
            int bits = bits_for(ntc);
            sort_pairs_i32(rkey.p, ks.p, ids.p, st.row_idx.p, na, bits, s);
            sort_pairs_i32(ckey.p, ks.p, ids.p, st.col_idx.p, na, bits, s);
            k_histogram<<<grid_for(na, kThreads), kThreads, 0, s>>>(rkey.p, na, rcnt.p);
            DH2_CHECK_LAUNCH("k_histogram");
            k_histogram<<<grid_for(na, kThreads), kThreads, 0, s>>>(ckey.p, na, ccnt.p);
            DH2_CHECK_LAUNCH("k_histogram");
        }
        exclusive_scan_i32(rcnt.p, st.row_ptr.p, ntc + 1, s);
        exclusive_scan_i32(ccnt.p, st.col_ptr.p, ntc + 1, s);
        st.active.alloc(ntc);
        k_active_seed<<<grid_for(ntc, kThreads), kThreads, 0, s>>>(rcnt.p, ccnt.p, ntc, st.active.p);
        DH2_CHECK_LAUNCH("k_active_seed");
    }
    std::vector<int32_t> tcb_h = st.tc_base.to_host(s);
    auto tc_of_level = [&](int l) -> int32_t {
        return l < nlev ? tcb_h[tr.level_start[l]] : (int32_t)ntc;
    };
    for (int l = 0; l + 1 < nlev; ++l) {
        int32_t b = tc_of_level(l), e = tc_of_level(l + 1);
        if (e > b) {
            k_active_close<<<grid_for(e - b, kThreads), kThreads, 0, s>>>(
                b, e, st.tc_cluster.p, st.tc_base.p, tr.son0.p, tr.son1.p, st.sd.p + st.dir_off[l],
                st.active.p);
            DH2_CHECK_LAUNCH("k_active_close");
        }
    }
    {
        DBuf<int32_t> a32(ntc), pos(ntc);
        k_to_i32<<<grid_for(ntc, kThreads), kThreads, 0, s>>>(st.active.p, ntc, a32.p);
        DH2_CHECK_LAUNCH("k_to_i32");
        st.nactive = exclusive_scan_i32(a32.p, pos.p, ntc, s);
        st.aidx.alloc(ntc);
        st.alist.alloc(st.nactive);
        st.a_t.alloc(st.nactive);
        st.a_c.alloc(st.nactive);
        k_active_lists<<<grid_for(ntc, kThreads), kThreads, 0, s>>>(
            st.active.p, pos.p, ntc, st.tc_cluster.p, st.tc_base.p, st.aidx.p, st.alist.p, st.a_t.p,
            st.a_c.p);
        DH2_CHECK_LAUNCH("k_active_lists");
        std::vector<int32_t> pos_h = pos.to_host(s);
        std::vector<int8_t> act_h = st.active.to_host(s);
        st.alevel_start.assign(nlev + 1, 0);
        for (int l = 0; l <= nlev; ++l) {
            int32_t b = tc_of_level(l);
            st.alevel_start[l] = b < ntc ? pos_h[b] : (int32_t)st.nactive;
        }
        (void)act_h;
    }
    DH2_CHECK_CUDA(cudaStreamSynchronize(s));
}

}  // namespace dh2
