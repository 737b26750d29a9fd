// LP relaxation: subgradient by sort + divide and conquer, projected subgradient.
//
// Section 6 of the paper (Eq. 18-20), Appendix D (reformulation), Appendix E
// (divide and conquer) and Algorithm 3, Potts model.
//
// For label i the pixels of every image are ranked by descending y(i), ties by
// ascending pixel index.  With B = ceil(log2 n) levels, at level l the node of
// a pixel is rank >> (B - l) and it lies in the right child when bit B-l-1 of
// its rank is set.  Each node's lattice is the global lattice restricted to
// the vertices its own points touch: a "tagged vertex" (label, vertex, node).
// All tagged vertices of a level are found without hashing: the incidence
// list (label, point, corner) is sorted once by (label, vertex, rank); at any
// level the entries of one tagged vertex are then a contiguous run, and the
// blur neighbour (label, v +- w_j, node) is the run of vertex v +- w_j whose
// ranks fall in the node, found by binary search inside that vertex's group.
// Per level: splat the right-child indicator into the runs, d+1 Jacobi blur
// passes over the runs, slice at the left-child points into U.
// Finally G = phi + 2U - c and S_LP = <y, G>.
#include <cub/device/device_segmented_radix_sort.cuh>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace {

inline unsigned nb(int64_t work, int threads) { return (unsigned)((work + threads - 1) / threads); }

inline int ceil_log2(int64_t n) {
    int b = 0;
    while ((1ll << b) < n) ++b;
    return b;
}

// Sort key of a column value: ascending keys = descending values (-0 is
// folded into +0 first, so equal values get equal keys and keep pixel order).
__device__ __forceinline__ uint32_t desc_key(float v) {
    const uint32_t b = __float_as_uint(v + 0.0f);
    const uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // ascending order of the floats
    return ~asc;
}

// keys[i][a] = key of y_a(i), vals[i][a] = a
__global__ void k_lp_transpose(const float *__restrict__ Y, int64_t n, int L, uint32_t *__restrict__ keys,
                               int32_t *__restrict__ vals, int *status) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n * L) return;
    const int64_t a = dcrf_div(q, L, n * L);
    const int i = (int)(q - a * L);
    float v = Y[q];
    if (!isfinite(v)) dcrf_flag(status, DCRF_E_NONFINITE);
    keys[(int64_t)i * n + a] = desc_key(v);
    vals[(int64_t)i * n + a] = (int32_t)a;
}

// Tree columns (Appendix F): keys[t][a] = y_a(T_t) = sum of y_a(i) over the
// labels i of subtree t (bit i of mask[t]), in label order; vals[t][a] = a
__global__ void k_lp_columns(const float *__restrict__ Y, int64_t n, int L, int C, const uint64_t *__restrict__ mask,
                             uint32_t *__restrict__ keys, int32_t *__restrict__ vals, int *status) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n * C) return;
    const int64_t a = dcrf_div(q, C, n * C);
    const int t = (int)(q - a * C);
    const uint64_t mk = mask[t];
    float v = 0.f;
    for (int i = 0; i < L; ++i)
        if ((mk >> i) & 1ull) v += Y[a * L + i];
    if (!isfinite(v)) dcrf_flag(status, DCRF_E_NONFINITE);
    keys[(int64_t)t * n + a] = desc_key(v);
    vals[(int64_t)t * n + a] = (int32_t)a;
}

// seg offsets for (label, image): begin = i*n + off[b]
__global__ void k_lp_segments(const int64_t *__restrict__ off, int batch, int L, int64_t n,
                              int64_t *__restrict__ begin, int64_t *__restrict__ end) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= L * batch) return;
    const int i = s / batch, b = s - i * batch;
    begin[s] = (int64_t)i * n + off[b];
    end[s] = (int64_t)i * n + off[b + 1];
}

// rankpos[i][a] = position p of a in label i's sorted list (global within the label row)
__global__ void k_lp_inverse(const int32_t *__restrict__ perm, int64_t n, int L, int32_t *__restrict__ inv) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n * L) return;
    const int64_t i = dcrf_div(q, (int)n, n * L);
    inv[i * n + perm[q]] = (int32_t)(q - i * n);
}

// Entries in (label, position, corner) order: key = vertex (the entries of
// one (label, image) are sorted by it, stably).
__global__ void k_lp_entries(const int32_t *__restrict__ perm, int64_t n, int L, int d1,
                             const int32_t *__restrict__ pvid, int64_t m, uint32_t *__restrict__ key,
                             int32_t *__restrict__ q_out) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t E = n * L * d1;
    if (q >= E) return;
    const int64_t ip = dcrf_div(q, d1, E);
    const int k = (int)(q - ip * d1);
    const int64_t i = dcrf_div(ip, (int)n, n * L);
    const int32_t a = perm[ip];
    const int v = pvid[(int64_t)a * d1 + k];
    (void)i;
    (void)m;
    key[q] = (uint32_t)(v < 0 ? 0 : v);
    q_out[q] = (int32_t)q;
}

// After the sort: per entry its vertex, rank, weight, and pos[q] = e.
__global__ void k_lp_unpack(const uint32_t *__restrict__ key_s, const int32_t *__restrict__ q_s, int64_t E,
                            int64_t n, int d1, int64_t m, const int32_t *__restrict__ perm,
                            const int64_t *__restrict__ point_off, int batch, const float *__restrict__ pbary,
                            int32_t *__restrict__ vid_s, int32_t *__restrict__ rank_s,
                            float *__restrict__ bary_s, int32_t *__restrict__ pos) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int64_t q = q_s[e];
    const int64_t ip = q / d1;
    const int k = (int)(q - ip * d1);
    const int64_t p = ip % n;
    const int32_t a = perm[ip];
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (point_off[mid] <= p) lo = mid; else hi = mid - 1;
    }
    (void)m;
    vid_s[e] = (int32_t)key_s[e];
    rank_s[e] = (int32_t)(p - point_off[lo]);
    bary_s[e] = pbary[(int64_t)a * d1 + k];
    pos[q] = (int32_t)e;
}

struct LevelArgs {
    const int32_t *vid_s;
    const int32_t *rank_s;
    const float *bary_s;
    const int32_t *vimg;      // [m]
    const int32_t *nlev;      // [batch] levels per image
    const int64_t *csr;       // [m+1] incidence offsets of every vertex (label-independent)
    const int32_t *nbr;       // [m][d1][2]
    const int32_t *local_from;  // [batch] first level handled by the shared-memory path
    int64_t E, n, m;
    int d1, level;
};

__device__ __forceinline__ bool entry_node(const LevelArgs &A, int64_t e, int32_t &node, int &bit) {
    const int v = A.vid_s[e];
    const int img = A.vimg[v];
    const int B = A.nlev[img];
    if (A.level >= B || A.level >= A.local_from[img]) return false;
    const int r = A.rank_s[e];
    node = r >> (B - A.level);
    bit = (r >> (B - A.level - 1)) & 1;
    return true;
}

__global__ void k_lp_flags(LevelArgs A, int32_t *__restrict__ flag) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= A.E) return;
    int f = 1;
    if (e > 0 && (e % (A.n * A.d1)) != 0 && A.vid_s[e] == A.vid_s[e - 1]) {
        int32_t n0, n1;
        int b0, b1;
        const bool a0 = entry_node(A, e, n0, b0), a1 = entry_node(A, e - 1, n1, b1);
        f = (a0 && a1 && n0 == n1) ? 0 : 1;
    }
    flag[e] = f;
}

__global__ void k_lp_splat(LevelArgs A, const int32_t *__restrict__ flag, const int32_t *__restrict__ rid,
                           float *__restrict__ val, int32_t *__restrict__ run_first) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= A.E) return;
    const int32_t r = rid[e] - 1;   // inclusive scan of run starts
    if (flag[e]) run_first[r] = (int32_t)e;
    int32_t node;
    int bit;
    if (entry_node(A, e, node, bit) && bit) atomicAdd(val + r, A.bary_s[e]);
}

// rnbr[r][j][side]: the run of (label, v -+ w_j, node) or -1.
__global__ void k_lp_neighbours(LevelArgs A, const int32_t *__restrict__ run_first, int64_t R,
                                const int32_t *__restrict__ rid, int32_t *__restrict__ rnbr) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int64_t e0 = run_first[r];
    int32_t node;
    int bit;
    const bool active = entry_node(A, e0, node, bit);
    const int v = A.vid_s[e0];
    const int64_t label_base = (e0 / (A.n * A.d1)) * (A.n * A.d1);
    const int B = A.nlev[A.vimg[v]];
    const int shift = B - A.level;
    for (int j = 0; j < A.d1; ++j) {
        for (int side = 0; side < 2; ++side) {
            int32_t out = -1;
            const int u = A.nbr[((int64_t)v * A.d1 + j) * 2 + side];
            if (active && u >= 0) {
                int64_t lo = label_base + A.csr[u], hi = label_base + A.csr[u + 1];
                const int64_t end = hi;
                while (lo < hi) {   // first entry with rank >> shift >= node
                    const int64_t mid = (lo + hi) >> 1;
                    if ((A.rank_s[mid] >> shift) < node) lo = mid + 1; else hi = mid;
                }
                if (lo < end && (A.rank_s[lo] >> shift) == node) out = rid[lo] - 1;
            }
            rnbr[(r * A.d1 + j) * 2 + side] = out;
        }
    }
}

__global__ void k_lp_blur(const float *__restrict__ in, float *__restrict__ out, const int32_t *__restrict__ rnbr,
                          int64_t R, int d1, int j) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int2 nbv = reinterpret_cast<const int2 *>(rnbr)[r * d1 + j];
    float v = 0.5f * in[r];
    if (nbv.x >= 0) v += 0.25f * in[nbv.x];
    if (nbv.y >= 0) v += 0.25f * in[nbv.y];
    out[r] = v;
}

// U[i][p] += ws0 * sum_k b_k val[run of (i, p, k)] for left-child positions.
__global__ void k_lp_slice(LevelArgs A, const int32_t *__restrict__ pos, const int32_t *__restrict__ rid,
                           const float *__restrict__ val, float ws0, float *__restrict__ U) {
    int64_t ip = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = A.E / A.d1;
    if (ip >= total) return;
    const int64_t e0 = pos[ip * A.d1];
    int32_t node;
    int bit;
    if (!entry_node(A, e0, node, bit) || bit) return;
    float acc = 0.f;
    for (int k = 0; k < A.d1; ++k) {
        const int64_t e = pos[ip * A.d1 + k];
        acc += A.bary_s[e] * val[rid[e] - 1];
    }
    U[ip] += ws0 * acc;
}

__global__ void k_lp_csr_count(const int32_t *__restrict__ pvid, int64_t count, unsigned *__restrict__ cnt) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < count) {
        const int v = pvid[q];
        if (v >= 0) atomicAdd(cnt + v, 1u);
    }
}

__global__ void k_lp_combine(const float *__restrict__ phi, const float *__restrict__ Y, const float *__restrict__ U,
                             const int32_t *__restrict__ inv, const float *__restrict__ c, int64_t n, int L,
                             const int64_t *__restrict__ off, int batch, float *__restrict__ G,
                             double *__restrict__ energy) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double part = 0.0;
    int img = -1;
    if (q < n * L) {
        const int64_t a = dcrf_div(q, L, n * L);
        const int i = (int)(q - a * L);
        const float g = phi[q] + 2.f * U[(int64_t)i * n + inv[(int64_t)i * n + a]] - c[a];
        G[q] = g;
        part = (double)Y[q] * g;
        int lo = 0, hi = batch - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= a) lo = mid; else hi = mid - 1;
        }
        img = lo;
    }
    if (energy) {
        // one atomic per warp when the warp lies in one image
        const int lane = threadIdx.x & 31;
        const int img0 = __shfl_sync(0xffffffffu, img, 0);
        const bool uni = __all_sync(0xffffffffu, img == img0 || img < 0);
        if (uni) {
            double sum = part;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
            if (lane == 0 && img0 >= 0) atomicAdd(energy + img0, sum);
        } else if (img >= 0) {
            atomicAdd(energy + img, part);
        }
    }
}

// Tree combine (Appendix F): G_a(k) = phi_a(k) + sum over subtrees t containing
// k of w_t (2 U_t(a) - c_a); energy[b] += <y, G> over image b
__global__ void k_lp_combine_tree(const float *__restrict__ phi, const float *__restrict__ Y,
                                  const float *__restrict__ U, const int32_t *__restrict__ inv,
                                  const float *__restrict__ c, int64_t n, int L, int C,
                                  const uint64_t *__restrict__ mask, const float *__restrict__ wt,
                                  const int64_t *__restrict__ off, int batch, float *__restrict__ G,
                                  double *__restrict__ energy) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double part = 0.0;
    int img = -1;
    if (q < n * L) {
        const int64_t a = dcrf_div(q, L, n * L);
        const int k = (int)(q - a * L);
        float g = phi[q];
        for (int t = 0; t < C; ++t)
            if ((mask[t] >> k) & 1ull) g += wt[t] * (2.f * U[(int64_t)t * n + inv[(int64_t)t * n + a]] - c[a]);
        G[q] = g;
        part = (double)Y[q] * g;
        int lo = 0, hi = batch - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= a) lo = mid; else hi = mid - 1;
        }
        img = lo;
    }
    if (energy) {
        const int lane = threadIdx.x & 31;
        const int img0 = __shfl_sync(0xffffffffu, img, 0);
        const bool uni = __all_sync(0xffffffffu, img == img0 || img < 0);
        if (uni) {
            double sum = part;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
            if (lane == 0 && img0 >= 0) atomicAdd(energy + img0, sum);
        } else if (img >= 0) {
            atomicAdd(energy + img, part);
        }
    }
}

__global__ void k_lp_c(int64_t n, const float *const *ones, const float *w, int nk, float sumw, float *c) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    float s = 0.f;
    for (int m = 0; m < nk; ++m) s += w[m] * ones[m][a];
    s -= sumw;
    c[a] = s > 0.f ? s : 0.f;
}

// Euclidean projection of one row onto the simplex by Michelot's active-set
// iteration: tau = (sum_{active} v - 1)/|active|, drop v_i <= tau, repeat.
template <int LP>
__global__ void k_project(const float *__restrict__ V, int64_t n, int L, const float *__restrict__ G,
                          const double *__restrict__ step, const int64_t *__restrict__ off, int batch,
                          float *__restrict__ Y) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    float beta = 0.f;
    if (G) {
        int lo = 0, hi = batch - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= a) lo = mid; else hi = mid - 1;
        }
        beta = (float)step[lo];
    }
    float v[LP];
    bool act[LP];
    float vmax = -INFINITY;
#pragma unroll
    for (int i = 0; i < LP; ++i) {
        v[i] = i < L ? V[a * L + i] - (G ? beta * G[a * L + i] : 0.f) : 0.f;
        act[i] = i < L;
        if (i < L) vmax = fmaxf(vmax, v[i]);
    }
    // the projection is unchanged by a shift of v; shifting by max v keeps
    // tau small, so that v - tau does not cancel for large inputs
#pragma unroll
    for (int i = 0; i < LP; ++i) v[i] -= vmax;
    float tau = 0.f;
    for (int it = 0; it <= L; ++it) {
        float s = 0.f;
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < LP; ++i)
            if (act[i]) { s += v[i]; ++cnt; }
        tau = (s - 1.f) / (float)cnt;
        bool changed = false;
#pragma unroll
        for (int i = 0; i < LP; ++i)
            if (act[i] && v[i] <= tau) { act[i] = false; changed = true; }
        if (!changed) break;
    }
#pragma unroll
    for (int i = 0; i < LP; ++i)
        if (i < L) Y[a * L + i] = act[i] ? v[i] - tau : 0.f;
}

dcrf_status launch_project(const float *V, int64_t n, int L, const float *G, const double *step,
                           const int64_t *off, int batch, float *Y, cudaStream_t s) {
    if (n == 0) return DCRF_OK;
    ProfScope ps(P_LP_PROJECT, s);
    if (L <= 8) k_project<8><<<nb(n, 128), 128, 0, s>>>(V, n, L, G, step, off, batch, Y);
    else if (L <= 24) k_project<24><<<nb(n, 128), 128, 0, s>>>(V, n, L, G, step, off, batch, Y);
    else k_project<64><<<nb(n, 128), 128, 0, s>>>(V, n, L, G, step, off, batch, Y);
    DCRF_LAUNCHED();
    return DCRF_OK;
}

// Deep levels in shared memory.  Once a node has at most kLocalP points, one
// block takes kLocalP consecutive positions of one (label, image): whole nodes.
// Its tagged vertices (node, vertex) go into a shared-memory hash table, the
// right-child indicator is splatted, the d+1 Jacobi passes run between two
// shared arrays, and the left-child points slice their sums into U.
constexpr int kLocalP = 128;            // positions per block
constexpr int kLocalBits = 11;
constexpr int kLocalSlots = 1 << kLocalBits;   // hash slots (load <= 0.75 for d+1 <= 6)
constexpr int kLocalThreads = 128;
constexpr uint32_t kLocalEmpty = 0xFFFFFFFFu;
constexpr int kLocalVertBits = 21;      // local vertex ids below 2^21

struct LocalBlock {
    int32_t label, image;
    int32_t p0;        // first position (rank) of the block within the image
};

struct LocalArgs {
    const LocalBlock *blocks;
    const int32_t *perm;          // [L][n]
    const int32_t *pvid;          // [n][d1]
    const float *pbary;
    const int32_t *nbr;           // [m][d1][2]
    const int64_t *point_off;     // [batch+1]
    const int64_t *vert_off;      // [batch+1]
    const int32_t *nlev;          // [batch]
    float *U;                     // [L][n] by position
    int64_t n;
    int d1, level;
    float ws0;
};

__device__ __forceinline__ uint32_t local_hash(uint32_t k) { return (k * 0x9E3779B1u) >> (32 - kLocalBits); }

__device__ __forceinline__ int local_insert(uint32_t *hkey, uint32_t key) {
    uint32_t h = local_hash(key);
    for (int probe = 0; probe < kLocalSlots; ++probe) {
        const int slot = (int)((h + probe) & (kLocalSlots - 1));
        const uint32_t prev = atomicCAS(hkey + slot, kLocalEmpty, key);
        if (prev == kLocalEmpty || prev == key) return slot;
    }
    return -1;
}

__device__ __forceinline__ int local_find(const uint32_t *hkey, uint32_t key) {
    uint32_t h = local_hash(key);
    for (int probe = 0; probe < kLocalSlots; ++probe) {
        const int slot = (int)((h + probe) & (kLocalSlots - 1));
        const uint32_t cur = hkey[slot];
        if (cur == key) return slot;
        if (cur == kLocalEmpty) return -1;
    }
    return -1;
}

__global__ void __launch_bounds__(kLocalThreads) k_lp_local(LocalArgs A) {
    extern __shared__ uint32_t lsm[];
    uint32_t *hkey = lsm;
    float *val = reinterpret_cast<float *>(lsm + kLocalSlots);
    float *tmp = val + kLocalSlots;
    uint16_t *occ = reinterpret_cast<uint16_t *>(tmp + kLocalSlots);   // occupied slots, compacted
    __shared__ int wsum[kLocalThreads / 32];
    const LocalBlock blk = A.blocks[blockIdx.x];
    const int b = blk.image;
    const int64_t off = A.point_off[b];
    const int64_t nb_pts = A.point_off[b + 1] - off;
    const int64_t voff = A.vert_off[b];
    const int sh = A.nlev[b] - A.level;          // node = rank >> sh
    const int p_end = (int)((int64_t)blk.p0 + kLocalP < nb_pts ? (int64_t)blk.p0 + kLocalP : nb_pts);
    const int node0 = blk.p0 >> sh;
    const int32_t *perm = A.perm + (int64_t)blk.label * A.n + off;
    for (int i = threadIdx.x; i < kLocalSlots; i += kLocalThreads) {
        hkey[i] = kLocalEmpty;
        val[i] = 0.f;
    }
    __syncthreads();
    // insert every (node, corner vertex); splat the right child's indicator.
    // Eight entries per thread per step: their global loads are issued first.
    const int count = (p_end - blk.p0) * A.d1;
    constexpr int kB = 8;
    for (int q0 = threadIdx.x; q0 < count; q0 += kB * kLocalThreads) {
        int vv[kB];
        float ww[kB];
        int pp[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int q = q0 + u * kLocalThreads;
            vv[u] = -1;
            if (q < count) {
                const int p = blk.p0 + q / A.d1;
                const int k = q - (q / A.d1) * A.d1;
                const int a = perm[p];
                pp[u] = p;
                vv[u] = A.pvid[(int64_t)a * A.d1 + k];
                ww[u] = A.pbary[(int64_t)a * A.d1 + k];
            }
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            if (vv[u] < 0) continue;
            const int p = pp[u];
            const uint32_t key = ((uint32_t)((p >> sh) - node0) << kLocalVertBits) | (uint32_t)(vv[u] - voff);
            const int slot = local_insert(hkey, key);
            if (slot >= 0 && ((p >> (sh - 1)) & 1)) atomicAdd(val + slot, ww[u]);
        }
    }
    __syncthreads();
    // compact the occupied slots (thread t scans slots [t S, t S + S) in order;
    // block-wide exclusive scan of the counts): the passes visit only those
    constexpr int kPer = kLocalSlots / kLocalThreads;
    int mine = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) mine += hkey[threadIdx.x * kPer + i] != kLocalEmpty;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int base = incl - mine, nocc = 0;
#pragma unroll
    for (int w = 0; w < kLocalThreads / 32; ++w) {
        if (w < wid) base += wsum[w];
        nocc += wsum[w];
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int slot = threadIdx.x * kPer + i;
        if (hkey[slot] != kLocalEmpty) occ[base++] = (uint16_t)slot;
    }
    __syncthreads();
    // d+1 Jacobi passes along w_j over the occupied slots, absent neighbours
    // read as 0; eight slots per thread per step so that their neighbour-table
    // loads are in flight together
    for (int j = 0; j < A.d1; ++j) {
        for (int s0 = threadIdx.x; s0 < nocc; s0 += kB * kLocalThreads) {
            uint32_t kk[kB];
            int2 nbv[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int i = s0 + u * kLocalThreads;
                const int slot = i < nocc ? occ[i] : 0;
                kk[u] = i < nocc ? hkey[slot] : kLocalEmpty;
                nbv[u] = make_int2(-1, -1);
                if (kk[u] != kLocalEmpty) {
                    const int64_t v = voff + (kk[u] & ((1u << kLocalVertBits) - 1));
                    nbv[u] = reinterpret_cast<const int2 *>(A.nbr)[v * A.d1 + j];
                }
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int i = s0 + u * kLocalThreads;
                if (i >= nocc) continue;
                const int slot = occ[i];
                float r = 0.f;
                if (kk[u] != kLocalEmpty) {
                    const uint32_t nodebits = kk[u] & ~((1u << kLocalVertBits) - 1);
                    r = 0.5f * val[slot];
                    if (nbv[u].x >= 0) {
                        const int s2 = local_find(hkey, nodebits | (uint32_t)(nbv[u].x - voff));
                        if (s2 >= 0) r += 0.25f * val[s2];
                    }
                    if (nbv[u].y >= 0) {
                        const int s2 = local_find(hkey, nodebits | (uint32_t)(nbv[u].y - voff));
                        if (s2 >= 0) r += 0.25f * val[s2];
                    }
                }
                tmp[slot] = r;
            }
        }
        __syncthreads();
        float *t = val;
        val = tmp;
        tmp = t;
    }
    // slice at the left child's points
    float *U = A.U + (int64_t)blk.label * A.n + off;
    for (int p = blk.p0 + threadIdx.x; p < p_end; p += kLocalThreads) {
        if ((p >> (sh - 1)) & 1) continue;
        const int a = perm[p];
        const uint32_t lnode = (uint32_t)((p >> sh) - node0);
        float acc = 0.f;
        for (int k = 0; k < A.d1; ++k) {
            const int v = A.pvid[(int64_t)a * A.d1 + k];
            if (v < 0) continue;
            const int slot = local_find(hkey, (lnode << kLocalVertBits) | (uint32_t)(v - voff));
            if (slot >= 0) acc += A.pbary[(int64_t)a * A.d1 + k] * val[slot];
        }
        U[p] += A.ws0 * acc;
    }
}

// Reusable workspace of the subgradient for one set of lattices.
struct LpWork {
    cudaStream_t s;
    Scratch sc;
    const dcrf_lattice *lats = nullptr;
    int nk = 0, L = 0, batch = 0;
    int C = 0;                        // sorted columns: the labels (Potts) or the subtrees (tree metric)
    uint64_t *cmask = nullptr;        // [C] label sets of the subtrees (tree metric only)
    float *cw = nullptr;              // [C] subtree weights c_T
    int64_t n = 0;
    float sumw = 0.f;
    float ws0[DCRF_MAX_KERNELS];
    int64_t *off_d = nullptr, *seg_b = nullptr, *seg_e = nullptr;
    int32_t *nlev_d = nullptr;
    int32_t *local_from_d[DCRF_MAX_KERNELS] = {};
    std::vector<int32_t> nlev_h;
    std::vector<std::vector<int32_t>> local_from_h;
    LocalBlock *lblocks = nullptr;
    size_t lblocks_cap = 0;
    int maxlev = 0;
    float *c = nullptr;
    uint32_t *keys = nullptr, *keys2 = nullptr, *keys3 = nullptr;
    int32_t *vals = nullptr, *vals2 = nullptr, *perm = nullptr, *inv = nullptr;
    std::vector<int64_t> colseg;      // host [C * batch + 1]: segments (column, image) of the sorted columns
    std::vector<int64_t> entseg[DCRF_MAX_KERNELS];   // host: segments (column, image) of the entries
    bool cub_sort = false;            // DCRF_LP_SORT=cub: CUB's radix sorts (a test comparator)
    float *U = nullptr;
    int64_t *csr[DCRF_MAX_KERNELS] = {};
    int64_t Emax = 0;
    uint32_t *ekey = nullptr, *ekey2 = nullptr, *ekey3 = nullptr;
    int32_t *eq = nullptr, *eq2 = nullptr, *eq3 = nullptr, *vid_s = nullptr, *rank_s = nullptr, *pos = nullptr;
    int64_t *eseg_b = nullptr, *eseg_e = nullptr;   // device segment bounds of the entries (CUB comparator)
    int32_t *flag = nullptr, *rid = nullptr, *run_first = nullptr, *rnbr = nullptr;
    float *bary_s = nullptr, *val = nullptr, *val2 = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;

    explicit LpWork(cudaStream_t st) : s(st), sc(st) {}

    // Potts: masks == nullptr (one column per label); tree metric: n_sub
    // subtrees with label masks and weights (host arrays).
    dcrf_status setup(const dcrf_lattice *lattices, const float *weights, int n_k, int L_, int n_sub = 0,
                      const uint64_t *masks = nullptr, const float *c_sub = nullptr) {
        DCRF_CHECK_STATUS(dcrf_check_lattices(lattices, n_k));
        if (!weights || L_ < 1 || L_ > DCRF_MAX_L) return DCRF_E_INVAL;
        lats = lattices;
        nk = n_k;
        L = L_;
        C = L;
        if (masks) {
            if (!c_sub || n_sub < 1) return DCRF_E_INVAL;
            const uint64_t all = L_ == 64 ? ~0ull : ((1ull << L_) - 1);
            for (int t = 0; t < n_sub; ++t)
                if (masks[t] == 0 || (masks[t] & ~all) || !(c_sub[t] >= 0.f) || !std::isfinite(c_sub[t]))
                    return DCRF_E_INVAL;
            C = n_sub;
            DCRF_CHECK_STATUS(sc.get(&cmask, (size_t)C));
            DCRF_CHECK_STATUS(sc.get(&cw, (size_t)C));
            DCRF_TRY(cudaMemcpyAsync(cmask, masks, C * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
            DCRF_TRY(cudaMemcpyAsync(cw, c_sub, C * sizeof(float), cudaMemcpyHostToDevice, s));
        }
        n = lattices[0]->n;
        batch = lattices[0]->batch;
        sumw = 0.f;
        for (int m = 0; m < nk; ++m) {
            if (!(weights[m] >= 0.f)) return DCRF_E_INVAL;
            sumw += weights[m];
            ws0[m] = (float)(weights[m] * lattices[m]->s0);
            Emax = std::max<int64_t>(Emax, n * C * (lattices[m]->d + 1));
        }
        if (Emax >= (1ll << 31)) return DCRF_E_INVAL;
        std::vector<int32_t> nlev(batch);
        for (int b = 0; b < batch; ++b) {
            nlev[b] = ceil_log2(lattices[0]->point_off[b + 1] - lattices[0]->point_off[b]);
            maxlev = std::max(maxlev, (int)nlev[b]);
        }
        DCRF_CHECK_STATUS(sc.get(&off_d, batch + 1));
        DCRF_CHECK_STATUS(sc.get(&nlev_d, batch));
        DCRF_CHECK_STATUS(sc.get(&seg_b, (size_t)C * batch));
        DCRF_CHECK_STATUS(sc.get(&seg_e, (size_t)C * batch));
        DCRF_TRY(cudaMemcpyAsync(off_d, lattices[0]->point_off.data(), (batch + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s));
        DCRF_TRY(cudaMemcpyAsync(nlev_d, nlev.data(), batch * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        nlev_h = nlev;
        // per lattice and image: the first level whose nodes fit one shared-memory block
        int pbits = 0;
        while ((1 << pbits) < kLocalP) ++pbits;
        local_from_h.assign(nk, std::vector<int32_t>(batch));
        size_t max_blocks = 1;
        for (int m = 0; m < nk; ++m) {
            for (int b = 0; b < batch; ++b) {
                const int64_t mb = lattices[m]->vert_off[b + 1] - lattices[m]->vert_off[b];
                const bool ok = lattices[m]->d + 1 <= 6 && mb < (1ll << kLocalVertBits);
                local_from_h[m][b] = ok ? std::max(0, nlev[b] - pbits) : nlev[b];
            }
            DCRF_CHECK_STATUS(sc.get(&local_from_d[m], (size_t)batch));
            DCRF_TRY(cudaMemcpyAsync(local_from_d[m], local_from_h[m].data(), batch * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, s));
        }
        for (int b = 0; b < batch; ++b) {
            const int64_t nb_ = lattices[0]->point_off[b + 1] - lattices[0]->point_off[b];
            max_blocks += (size_t)C * (size_t)((nb_ + kLocalP - 1) / kLocalP);
        }
        DCRF_CHECK_STATUS(sc.get(&lblocks, max_blocks));
        lblocks_cap = max_blocks;
        k_lp_segments<<<nb(C * batch, 128), 128, 0, s>>>(off_d, batch, C, n, seg_b, seg_e);
        DCRF_LAUNCHED();
        const size_t nl = (size_t)(n > 0 ? n : 1) * C;   // sorted columns
        DCRF_CHECK_STATUS(sc.get(&c, (size_t)(n > 0 ? n : 1)));
        DCRF_CHECK_STATUS(sc.get(&keys, nl));
        DCRF_CHECK_STATUS(sc.get(&keys2, nl));
        DCRF_CHECK_STATUS(sc.get(&keys3, nl));
        DCRF_CHECK_STATUS(sc.get(&vals, nl));
        DCRF_CHECK_STATUS(sc.get(&vals2, nl));
        DCRF_CHECK_STATUS(sc.get(&perm, nl));
        DCRF_CHECK_STATUS(sc.get(&inv, nl));
        DCRF_CHECK_STATUS(sc.get(&U, nl));
        const size_t ne = (size_t)(Emax > 0 ? Emax : 1);
        DCRF_CHECK_STATUS(sc.get(&ekey, ne));
        DCRF_CHECK_STATUS(sc.get(&ekey2, ne));
        DCRF_CHECK_STATUS(sc.get(&ekey3, ne));
        DCRF_CHECK_STATUS(sc.get(&eq, ne));
        DCRF_CHECK_STATUS(sc.get(&eq2, ne));
        DCRF_CHECK_STATUS(sc.get(&eq3, ne));
        // sort segments: every (column, image) of the sorted columns, and of
        // the entries (d+1 per position)
        const std::vector<int64_t> &po = lattices[0]->point_off;
        colseg.clear();
        for (int i = 0; i < C; ++i)
            for (int b = 0; b < batch; ++b) colseg.push_back((int64_t)i * n + po[b]);
        colseg.push_back((int64_t)C * n);
        for (int m = 0; m < nk; ++m) {
            entseg[m].clear();
            for (int64_t x : colseg) entseg[m].push_back(x * (lattices[m]->d + 1));
        }
        const char *srt = std::getenv("DCRF_LP_SORT");
        cub_sort = srt && std::strcmp(srt, "cub") == 0;
        DCRF_CHECK_STATUS(sc.get(&eseg_b, (size_t)C * batch));
        DCRF_CHECK_STATUS(sc.get(&eseg_e, (size_t)C * batch));
        DCRF_CHECK_STATUS(sc.get(&vid_s, ne));
        DCRF_CHECK_STATUS(sc.get(&rank_s, ne));
        DCRF_CHECK_STATUS(sc.get(&pos, ne));
        DCRF_CHECK_STATUS(sc.get(&flag, ne));
        DCRF_CHECK_STATUS(sc.get(&rid, ne));
        DCRF_CHECK_STATUS(sc.get(&run_first, ne));
        DCRF_CHECK_STATUS(sc.get(&bary_s, ne));
        DCRF_CHECK_STATUS(sc.get(&val, ne));
        DCRF_CHECK_STATUS(sc.get(&val2, ne));
        int dmax = 1;
        for (int m = 0; m < nk; ++m) dmax = std::max(dmax, lattices[m]->d + 1);
        DCRF_CHECK_STATUS(sc.get(&rnbr, ne * dmax * 2));
        if (cub_sort) {   // temp storage for the CUB sorts (the comparator path)
            size_t t1 = 0, t2 = 0;
            DCRF_TRY(cub::DeviceSegmentedRadixSort::SortPairs(nullptr, t1, keys, keys2, vals, perm, (int)nl,
                                                              C * batch, seg_b, seg_e, 0, 32, s));
            DCRF_TRY(cub::DeviceSegmentedRadixSort::SortPairs(nullptr, t2, ekey, ekey2, eq, eq2, (int)ne, C * batch,
                                                              eseg_b, eseg_e, 0, 32, s));
            tmp_bytes = std::max(t1, t2);
            char *t;
            DCRF_CHECK_STATUS(sc.get(&t, tmp_bytes));
            tmp = t;
        }
        // incidence offsets per vertex (label independent)
        for (int m = 0; m < nk; ++m) {
            const dcrf_lattice lat = lattices[m];
            unsigned *cnt;
            DCRF_CHECK_STATUS(sc.get(&cnt, (size_t)lat->m + 1));
            DCRF_CHECK_STATUS(sc.get(&csr[m], (size_t)lat->m + 1));
            DCRF_TRY(cudaMemsetAsync(cnt, 0, (lat->m + 1) * sizeof(unsigned), s));
            if (n > 0) {
                k_lp_csr_count<<<nb(n * (lat->d + 1), 256), 256, 0, s>>>(lat->pvid, n * (lat->d + 1), cnt);
                DCRF_LAUNCHED();
            }
            DCRF_CHECK_STATUS(dcrf_scan(cnt, csr[m], lat->m + 1, false, s));
        }
        // c_a
        const float *ones_h[DCRF_MAX_KERNELS];
        for (int m = 0; m < nk; ++m) ones_h[m] = lattices[m]->ones;
        const float **ones_d;
        float *w_d;
        DCRF_CHECK_STATUS(sc.get(&ones_d, nk));
        DCRF_CHECK_STATUS(sc.get(&w_d, nk));
        DCRF_TRY(cudaMemcpyAsync(ones_d, ones_h, nk * sizeof(float *), cudaMemcpyHostToDevice, s));
        DCRF_TRY(cudaMemcpyAsync(w_d, weights, nk * sizeof(float), cudaMemcpyHostToDevice, s));
        if (n > 0) {
            k_lp_c<<<nb(n, 256), 256, 0, s>>>(n, ones_d, w_d, nk, sumw, c);
            DCRF_LAUNCHED();
        }
        return DCRF_OK;
    }

    // G = phi + 2U - c; energy[b] += <y, G> over image b (energy zeroed by caller)
    dcrf_status subgrad(const float *phi, const float *Y, float *G, double *energy) {
        if (n == 0) return DCRF_OK;
        const int64_t nl = n * C;        // sorted columns x pixels
        {
            ProfScope ps(P_LP_SORT, s);
            if (cmask)
                k_lp_columns<<<nb(nl, 256), 256, 0, s>>>(Y, n, L, C, cmask, keys, vals, lats[0]->status);
            else
                k_lp_transpose<<<nb(nl, 256), 256, 0, s>>>(Y, n, L, keys, vals, lats[0]->status);
            DCRF_LAUNCHED();
            if (cub_sort) {
                size_t tb = tmp_bytes;
                DCRF_TRY(cub::DeviceSegmentedRadixSort::SortPairs(tmp, tb, keys, keys2, vals, perm, (int)nl,
                                                                  C * batch, seg_b, seg_e, 0, 32, s));
            } else {
                DCRF_CHECK_STATUS(dcrf_segsort(keys, vals, keys3, vals2, keys2, perm, colseg.data(), C * batch, 32,
                                               s));
            }
            k_lp_inverse<<<nb(nl, 256), 256, 0, s>>>(perm, n, C, inv);
            DCRF_LAUNCHED();
        }
        DCRF_TRY(cudaMemsetAsync(U, 0, nl * sizeof(float), s));
        for (int mm = 0; mm < nk; ++mm) {
            const dcrf_lattice lat = lats[mm];
            const int d1 = lat->d + 1;
            const int64_t E = nl * d1;
            const int64_t m = lat->m > 0 ? lat->m : 1;
            int keybits = 1;
            while (keybits < 32 && (uint64_t)m > (1ull << keybits)) ++keybits;
            {
                ProfScope ps(P_LP_SORT, s);
                k_lp_entries<<<nb(E, 256), 256, 0, s>>>(perm, n, C, d1, lat->pvid, m, ekey, eq);
                DCRF_LAUNCHED();
                if (cub_sort) {
                    std::vector<int64_t> eb(entseg[mm].begin(), entseg[mm].end() - 1),
                        ee(entseg[mm].begin() + 1, entseg[mm].end());
                    DCRF_TRY(cudaMemcpyAsync(eseg_b, eb.data(), eb.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
                    DCRF_TRY(cudaMemcpyAsync(eseg_e, ee.data(), ee.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
                    size_t tb = tmp_bytes;
                    DCRF_TRY(cub::DeviceSegmentedRadixSort::SortPairs(tmp, tb, ekey, ekey2, eq, eq2, (int)E, C * batch,
                                                                      eseg_b, eseg_e, 0, keybits, s));
                } else {
                    DCRF_CHECK_STATUS(dcrf_segsort(ekey, eq, ekey3, eq3, ekey2, eq2, entseg[mm].data(), C * batch,
                                                   keybits, s));
                }
                k_lp_unpack<<<nb(E, 256), 256, 0, s>>>(ekey2, eq2, E, n, d1, m, perm, off_d, batch, lat->pbary,
                                                       vid_s, rank_s, bary_s, pos);
                DCRF_LAUNCHED();
            }
            LevelArgs A;
            A.vid_s = vid_s;
            A.rank_s = rank_s;
            A.bary_s = bary_s;
            A.vimg = lat->vimg;
            A.nlev = nlev_d;
            A.csr = csr[mm];
            A.nbr = lat->nbr;
            A.E = E;
            A.n = n;
            A.m = m;
            A.d1 = d1;
            A.local_from = local_from_d[mm];
            for (int lev = 0; lev < maxlev; ++lev) {
                A.level = lev;
                // images whose nodes fit a shared-memory block at this level
                std::vector<LocalBlock> lb;
                bool any_global = false;
                for (int b = 0; b < batch; ++b) {
                    if (lev >= nlev_h[b]) continue;
                    if (lev >= local_from_h[mm][b]) {
                        const int64_t nb_ = lat->point_off[b + 1] - lat->point_off[b];
                        for (int i = 0; i < C; ++i)
                            for (int64_t p0 = 0; p0 < nb_; p0 += kLocalP) lb.push_back(LocalBlock{i, b, (int32_t)p0});
                    } else {
                        any_global = true;
                    }
                }
                if (!lb.empty()) {
                    DCRF_TRY(cudaMemcpyAsync(lblocks, lb.data(), lb.size() * sizeof(LocalBlock), cudaMemcpyHostToDevice, s));
                    LocalArgs la;
                    la.blocks = lblocks;
                    la.perm = perm;
                    la.pvid = lat->pvid;
                    la.pbary = lat->pbary;
                    la.nbr = lat->nbr;
                    la.point_off = off_d;
                    la.vert_off = lat->vert_off_d;
                    la.nlev = nlev_d;
                    la.U = U;
                    la.n = n;
                    la.d1 = d1;
                    la.level = lev;
                    la.ws0 = ws0[mm];
                    const size_t shm = (size_t)kLocalSlots * 14;   // key, value, value, occupied index
                    static bool attr = false;
                    if (!attr) {
                        DCRF_TRY(cudaFuncSetAttribute(k_lp_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
                        attr = true;
                    }
                    ProfScope ps(P_LP_LOCAL, s);
                    k_lp_local<<<(unsigned)lb.size(), kLocalThreads, shm, s>>>(la);
                    DCRF_LAUNCHED();
                    // the block list is read by the kernel before the next level's copy:
                    // copies and kernels on one stream run in order
                }
                if (!any_global) continue;
                {
                    ProfScope ps(P_LP_RUNS, s);
                    k_lp_flags<<<nb(E, 256), 256, 0, s>>>(A, flag);
                    DCRF_LAUNCHED();
                    DCRF_CHECK_STATUS(dcrf_scan(flag, rid, E, true, s));
                }
                // rid[e] = 1 + run of entry e; the number of runs is rid[E-1]
                int32_t last = 0;
                DCRF_TRY(cudaMemcpyAsync(&last, rid + E - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                DCRF_TRY(cudaStreamSynchronize(s));
                const int64_t R = (int64_t)last;
                DCRF_TRY(cudaMemsetAsync(val, 0, R * sizeof(float), s));
                {
                    ProfScope ps(P_LP_SPLAT, s);
                    k_lp_splat<<<nb(E, 256), 256, 0, s>>>(A, flag, rid, val, run_first);
                    DCRF_LAUNCHED();
                }
                {
                    ProfScope ps(P_LP_NEIGHBOURS, s);
                    k_lp_neighbours<<<nb(R, 128), 128, 0, s>>>(A, run_first, R, rid, rnbr);
                    DCRF_LAUNCHED();
                }
                float *in = val, *out = val2;
                for (int j = 0; j < d1; ++j) {
                    ProfScope ps(P_LP_BLUR, s);
                    k_lp_blur<<<nb(R, 256), 256, 0, s>>>(in, out, rnbr, R, d1, j);
                    DCRF_LAUNCHED();
                    std::swap(in, out);
                }
                {
                    ProfScope ps(P_LP_SLICE, s);
                    k_lp_slice<<<nb(nl, 256), 256, 0, s>>>(A, pos, rid, in, ws0[mm], U);
                    DCRF_LAUNCHED();
                }
            }
        }
        {
            ProfScope ps(P_LP_COMBINE, s);
            if (cmask)
                k_lp_combine_tree<<<nb(n * L, 256), 256, 0, s>>>(phi, Y, U, inv, c, n, L, C, cmask, cw, off_d,
                                                                  batch, G, energy);
            else
                k_lp_combine<<<nb(nl, 256), 256, 0, s>>>(phi, Y, U, inv, c, n, L, off_d, batch, G, energy);
            DCRF_LAUNCHED();
        }
        return DCRF_OK;
    }
};

__global__ void k_lp_beta0(const float *__restrict__ G, int64_t n, int L, const int64_t *__restrict__ off,
                           int batch, unsigned *__restrict__ maxdev) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    float mean = 0.f;
    for (int i = 0; i < L; ++i) mean += G[a * L + i];
    mean /= (float)L;
    float dev = 0.f;
    for (int i = 0; i < L; ++i) dev = fmaxf(dev, fabsf(G[a * L + i] - mean));
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= a) lo = mid; else hi = mid - 1;
    }
    atomicMax(maxdev + lo, __float_as_uint(dev));   // non-negative floats order as their bits
}

__global__ void k_lp_steps(const unsigned *__restrict__ maxdev, double beta0, int batch, double *__restrict__ b0) {
    for (int b = threadIdx.x; b < batch; b += blockDim.x) {
        if (beta0 > 0.0) { b0[b] = beta0; continue; }
        const float dv = __uint_as_float(maxdev[b]);
        b0[b] = dv > 0.f ? 0.1 / (double)dv : 0.1;
    }
}

__global__ void k_lp_scale(const double *__restrict__ b0, double factor, int batch, double *__restrict__ step) {
    for (int b = threadIdx.x; b < batch; b += blockDim.x) step[b] = b0[b] * factor;
}

// keep the best iterate per image: if e[b] < best[b] copy image b's rows
__global__ void k_lp_keep_best(const double *__restrict__ e, double *__restrict__ best, int batch,
                               int *__restrict__ take) {
    for (int b = threadIdx.x; b < batch; b += blockDim.x) {
        take[b] = e[b] < best[b];
        if (take[b]) best[b] = e[b];
    }
}

__global__ void k_lp_copy_rows(const float *__restrict__ src, float *__restrict__ dst, int64_t n, int L,
                               const int64_t *__restrict__ off, int batch, const int *__restrict__ take) {
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= n * L) return;
    const int64_t a = dcrf_div(q, L, n * L);
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= a) lo = mid; else hi = mid - 1;
    }
    if (!take || take[lo]) dst[q] = src[q];
}

}  // namespace

namespace {

dcrf_status lp_subgrad_impl(const float *unaries, const float *Y, const dcrf_lattice *lattices, const float *weights,
                            int n_kernels, int L, int n_sub, const uint64_t *masks, const float *c_sub, float *G,
                            double *energy, cudaStream_t s) {
    if (!unaries || !Y || !G) return DCRF_E_INVAL;
    LpWork W(s);
    DCRF_CHECK_STATUS(W.setup(lattices, weights, n_kernels, L, n_sub, masks, c_sub));
    double *e;
    DCRF_CHECK_STATUS(W.sc.get(&e, (size_t)W.batch));
    DCRF_TRY(cudaMemsetAsync(e, 0, W.batch * sizeof(double), s));
    DCRF_CHECK_STATUS(W.subgrad(unaries, Y, G, e));
    if (energy) {
        DCRF_TRY(cudaMemcpyAsync(energy, e, W.batch * sizeof(double), cudaMemcpyDeviceToHost, s));
        int h = 0;
        DCRF_TRY(cudaMemcpyAsync(&h, lattices[0]->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DCRF_TRY(cudaStreamSynchronize(s));
        if (h != 0) return (dcrf_status)h;
    }
    return DCRF_OK;
}

dcrf_status lp_solve_impl(const float *unaries, const dcrf_lattice *lattices, const float *weights, int n_kernels,
                          int L, int n_sub, const uint64_t *masks, const float *c_sub, int steps, double beta0,
                          float *Y, double *energies, cudaStream_t s) {
    if (!unaries || !Y || steps < 0) return DCRF_E_INVAL;
    LpWork W(s);
    DCRF_CHECK_STATUS(W.setup(lattices, weights, n_kernels, L, n_sub, masks, c_sub));
    if (W.n == 0) return DCRF_OK;
    const int batch = W.batch;
    const int64_t nl = W.n * L;
    float *G, *Yb;
    double *e, *best, *b0, *step;
    unsigned *maxdev;
    int *take;
    DCRF_CHECK_STATUS(W.sc.get(&G, (size_t)nl));
    DCRF_CHECK_STATUS(W.sc.get(&Yb, (size_t)nl));
    DCRF_CHECK_STATUS(W.sc.get(&e, (size_t)(steps + 1) * batch));
    DCRF_CHECK_STATUS(W.sc.get(&best, (size_t)batch));
    DCRF_CHECK_STATUS(W.sc.get(&b0, (size_t)batch));
    DCRF_CHECK_STATUS(W.sc.get(&step, (size_t)batch));
    DCRF_CHECK_STATUS(W.sc.get(&maxdev, (size_t)batch));
    DCRF_CHECK_STATUS(W.sc.get(&take, (size_t)batch));
    DCRF_TRY(cudaMemsetAsync(e, 0, (steps + 1) * batch * sizeof(double), s));
    DCRF_TRY(cudaMemsetAsync(maxdev, 0, batch * sizeof(unsigned), s));
    DCRF_CHECK_STATUS(W.subgrad(unaries, Y, G, e));
    DCRF_TRY(cudaMemcpyAsync(best, e, batch * sizeof(double), cudaMemcpyDeviceToDevice, s));
    DCRF_TRY(cudaMemcpyAsync(Yb, Y, nl * sizeof(float), cudaMemcpyDeviceToDevice, s));
    k_lp_beta0<<<nb(W.n, 256), 256, 0, s>>>(G, W.n, L, W.off_d, batch, maxdev);
    DCRF_LAUNCHED();
    k_lp_steps<<<1, 256, 0, s>>>(maxdev, beta0, batch, b0);
    DCRF_LAUNCHED();
    for (int t = 0; t < steps; ++t) {
        k_lp_scale<<<1, 256, 0, s>>>(b0, 1.0 / (1.0 + t), batch, step);
        DCRF_LAUNCHED();
        DCRF_CHECK_STATUS(launch_project(Y, W.n, L, G, step, W.off_d, batch, Y, s));
        double *et = e + (int64_t)(t + 1) * batch;
        DCRF_CHECK_STATUS(W.subgrad(unaries, Y, G, et));
        k_lp_keep_best<<<1, 256, 0, s>>>(et, best, batch, take);
        DCRF_LAUNCHED();
        k_lp_copy_rows<<<nb(nl, 256), 256, 0, s>>>(Y, Yb, W.n, L, W.off_d, batch, take);
        DCRF_LAUNCHED();
    }
    k_lp_copy_rows<<<nb(nl, 256), 256, 0, s>>>(Yb, Y, W.n, L, W.off_d, batch, nullptr);
    DCRF_LAUNCHED();
    if (energies) {
        DCRF_TRY(cudaMemcpyAsync(energies, e, (steps + 1) * batch * sizeof(double), cudaMemcpyDeviceToHost, s));
        int h = 0;
        DCRF_TRY(cudaMemcpyAsync(&h, lattices[0]->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DCRF_TRY(cudaStreamSynchronize(s));
        if (h != 0) return (dcrf_status)h;
    }
    return DCRF_OK;
}

}  // namespace

extern "C" dcrf_status dcrf_lp_subgrad(const float *unaries, const float *Y, const dcrf_lattice *lattices,
                                       const float *weights, int n_kernels, int L, float *G, double *energy,
                                       dcrf_stream stream) {
    return lp_subgrad_impl(unaries, Y, lattices, weights, n_kernels, L, 0, nullptr, nullptr, G, energy,
                           (cudaStream_t)stream);
}

extern "C" dcrf_status dcrf_lp_subgrad_tree(const float *unaries, const float *Y, const dcrf_lattice *lattices,
                                            const float *weights, int n_kernels, int L, int n_subtrees,
                                            const uint64_t *subtree_labels, const float *subtree_weights, float *G,
                                            double *energy, dcrf_stream stream) {
    if (!subtree_labels || !subtree_weights) return DCRF_E_INVAL;
    return lp_subgrad_impl(unaries, Y, lattices, weights, n_kernels, L, n_subtrees, subtree_labels,
                           subtree_weights, G, energy, (cudaStream_t)stream);
}

extern "C" dcrf_status dcrf_lp_solve(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                     int n_kernels, int L, int steps, double beta0, float *Y, double *energies,
                                     dcrf_stream stream) {
    return lp_solve_impl(unaries, lattices, weights, n_kernels, L, 0, nullptr, nullptr, steps, beta0, Y, energies,
                         (cudaStream_t)stream);
}

extern "C" dcrf_status dcrf_lp_solve_tree(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                          int n_kernels, int L, int n_subtrees, const uint64_t *subtree_labels,
                                          const float *subtree_weights, int steps, double beta0, float *Y,
                                          double *energies, dcrf_stream stream) {
    if (!subtree_labels || !subtree_weights) return DCRF_E_INVAL;
    return lp_solve_impl(unaries, lattices, weights, n_kernels, L, n_subtrees, subtree_labels, subtree_weights, steps,
                         beta0, Y, energies, (cudaStream_t)stream);
}

extern "C" dcrf_status dcrf_simplex_project(const float *V, int64_t n, int L, float *Y, dcrf_stream stream) {
    if (!V || !Y || n < 0 || L < 1 || L > DCRF_MAX_L) return DCRF_E_INVAL;
    return launch_project(V, n, L, nullptr, nullptr, nullptr, 1, Y, (cudaStream_t)stream);
}
