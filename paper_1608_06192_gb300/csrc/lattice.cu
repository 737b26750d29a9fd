// Permutohedral lattice: features, GPU hash-table build, filter and adjoint.
//
// The paper computes sum_b k(f_a, f_b) v_b with the permutohedral-lattice
// filter it cites (Section 3 "Filter-based Method", Eq. 6; Appendix A), not
// normalised.  Lattice conventions (scale, elevation, enclosing simplex,
// blur, output scale), shared with the CPU oracle:
//   c_j   = f_j * alpha / sqrt((j+1)(j+2)),  alpha = (d+1) sqrt(2/3)
//   x     = Helmert elevation onto sum(x) = 0 (FP64, one rounding per op)
//   m_i   = rint(x_i / (d+1)), rank correction, barycentric weights
//   blur  = d+1 Jacobi passes [1/4, 1/2, 1/4] along w_j = (d+1) e_j - 1
//   s0    = (2 pi)^{d/2} alpha^d / (d+1)^{d - 1/2}

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "common.cuh"

// ---------------------------------------------------------------------------
// host helpers

extern "C" const char *dcrf_status_string(int status) {
    switch (status) {
    case DCRF_OK: return "ok";
    case DCRF_E_INVAL: return "invalid argument";
    case DCRF_E_NOMEM: return "device allocation failed";
    case DCRF_E_CUDA: return "CUDA error";
    case DCRF_E_TABLE_FULL: return "lattice hash table full";
    case DCRF_E_KEY_RANGE: return "lattice coordinate outside the packed key range";
    case DCRF_E_TIMEOUT: return "bounded device wait expired";
    case DCRF_E_NONFINITE: return "non-finite value";
    case DCRF_E_SCRATCH: return "request exceeds the fixed scratch of dcrf_filter_static";
    default: return "unknown status";
    }
}

extern "C" int dcrf_version(void) { return 1; }

std::vector<Chunk> make_chunks(const std::vector<int64_t> &off, int size) {
    std::vector<Chunk> out;
    for (size_t b = 0; b + 1 < off.size(); ++b) {
        for (int64_t s = off[b]; s < off[b + 1]; s += size) {
            int64_t e = s + size < off[b + 1] ? s + size : off[b + 1];
            out.push_back(Chunk{s, (int32_t)(e - s), (int32_t)b});
        }
    }
    return out;
}

int dcrf_round4(int L) { return (L + 3) & ~3; }

dcrf_status dcrf_check_lattices(const dcrf_lattice *lats, int n_k) {
    if (!lats || n_k < 1 || n_k > DCRF_MAX_KERNELS) return DCRF_E_INVAL;
    for (int i = 0; i < n_k; ++i) {
        if (!lats[i]) return DCRF_E_INVAL;
        if (lats[i]->n != lats[0]->n || lats[i]->batch != lats[0]->batch) return DCRF_E_INVAL;
        for (int b = 0; b <= lats[0]->batch; ++b)
            if (lats[i]->point_off[b] != lats[0]->point_off[b]) return DCRF_E_INVAL;
    }
    return DCRF_OK;
}

static inline unsigned blocks_for(int64_t work, int threads) {
    return (unsigned)((work + threads - 1) / threads);
}

// ---------------------------------------------------------------------------
// a1: features (Appendix G): (x/ta, y/ta, r/tb, g/tb, b/tb) and (x, y)/tg.

__global__ void k_features(const float *__restrict__ rgb, const int64_t *__restrict__ off,
                           const int32_t *__restrict__ widths, int batch, int64_t n, float ta,
                           float tb, float tg, float *__restrict__ fb, float *__restrict__ fs) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= a) lo = mid; else hi = mid - 1;
    }
    int64_t local = a - off[lo];
    int w = widths[lo];
    float x = (float)(local % w);
    float y = (float)(local / w);
    if (fb) {
        fb[a * 5 + 0] = __fdiv_rn(x, ta);
        fb[a * 5 + 1] = __fdiv_rn(y, ta);
        fb[a * 5 + 2] = __fdiv_rn(rgb[a * 3 + 0], tb);
        fb[a * 5 + 3] = __fdiv_rn(rgb[a * 3 + 1], tb);
        fb[a * 5 + 4] = __fdiv_rn(rgb[a * 3 + 2], tb);
    }
    if (fs) {
        fs[a * 2 + 0] = __fdiv_rn(x, tg);
        fs[a * 2 + 1] = __fdiv_rn(y, tg);
    }
}

extern "C" dcrf_status dcrf_features(const float *rgb, const int32_t *widths, const int32_t *heights,
                                     int batch, float theta_alpha, float theta_beta,
                                     float theta_gamma, float *f_bil, float *f_sp,
                                     dcrf_stream stream) {
    if (!widths || !heights || batch < 1 || (!f_bil && !f_sp)) return DCRF_E_INVAL;
    if (!(theta_alpha > 0.f) || !(theta_beta > 0.f) || !(theta_gamma > 0.f)) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> off(batch + 1, 0);
    for (int b = 0; b < batch; ++b) {
        if (widths[b] < 0 || heights[b] < 0) return DCRF_E_INVAL;
        off[b + 1] = off[b] + (int64_t)widths[b] * heights[b];
    }
    if (off[batch] == 0) return DCRF_OK;           // every image empty
    if (!rgb) return DCRF_E_INVAL;
    Scratch sc(s);
    int64_t *off_d;
    int32_t *w_d;
    DCRF_CHECK_STATUS(sc.get(&off_d, batch + 1));
    DCRF_CHECK_STATUS(sc.get(&w_d, batch));
    DCRF_TRY(cudaMemcpyAsync(off_d, off.data(), (batch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DCRF_TRY(cudaMemcpyAsync(w_d, widths, batch * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    int64_t n = off[batch];
    k_features<<<blocks_for(n, 256), 256, 0, s>>>(rgb, off_d, w_d, batch, n, theta_alpha, theta_beta,
                                                  theta_gamma, f_bil, f_sp);
    DCRF_LAUNCHED();
    return DCRF_OK;
}

// ---------------------------------------------------------------------------
// a2: lattice build

struct EmbedParams {
    double sig[DCRF_MAX_D];
    int batch;
};

__device__ __forceinline__ int find_image(const int64_t *__restrict__ off, int batch, int64_t a) {
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= a) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Packs coordinates 0..D-1 of a vertex; false when a field leaves its range.
template <int D>
__device__ __forceinline__ bool pack_key(const long long *coord, uint64_t &key) {
    constexpr int bits = (64 / D) > 32 ? 32 : (64 / D);
    const long long bias = 1ll << (bits - 1);
    const long long top = (bits == 32) ? 0xFFFFFFFFll : ((1ll << bits) - 1);
    key = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        long long f = coord[i] + bias;
        if (f < 0 || f >= top) return false;
        key |= (uint64_t)f << (bits * i);
    }
    return true;
}

template <int D>
__global__ void k_embed_insert(const float *__restrict__ feat, int64_t n, EmbedParams P,
                               const int64_t *__restrict__ point_off,
                               const int64_t *__restrict__ tab_base,
                               const int64_t *__restrict__ tab_mask,
                               unsigned long long *__restrict__ table, int64_t *__restrict__ pslot,
                               float *__restrict__ pbary, int *__restrict__ status, uint64_t max_probe) {
    constexpr int D1 = D + 1;
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    int img = find_image(point_off, P.batch, a);

    // scale and elevate (one IEEE rounding per operation, no contraction)
    double c[D];
#pragma unroll
    for (int j = 0; j < D; ++j) c[j] = __dmul_rn((double)feat[a * D + j], P.sig[j]);
    double x[D1];
    double sm = 0.0;
#pragma unroll
    for (int i = D; i >= 1; --i) {
        x[i] = __dsub_rn(sm, __dmul_rn((double)i, c[i - 1]));
        sm = __dadd_rn(sm, c[i - 1]);
    }
    x[0] = sm;

    // nearest remainder-0 point: m_i = rint(x_i / (d+1)) and
    // delta_i = x_i - (d+1) m_i, as the correctly rounded quotient gives them,
    // without the FP64 division where that is provable (FP64 throughput bounds
    // this kernel).  With k = rint(x RN(1/(d+1))) and rem = RN(x - (d+1) k),
    // |RN(x/(d+1)) - k| <= |rem|/(d+1) + 2^-53 (|k| + 2) < |rem|/(d+1) + 2^-13
    // for |k| < 2^40 (larger k fail the 1e12 range check below whichever way
    // they are found), so when |rem| <= 0.499 (d+1) the quotient rounds to k
    // and rem is the delta the division would give; otherwise (near a tie,
    // or not finite) the division decides.
    const double inv = 1.0 / (double)D1;
    constexpr double thr = 0.499 * D1;
    long long mi[D1];
    double delta[D1];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < D1; ++i) {
        double q = rint(__dmul_rn(x[i], inv));
        double rem = __dsub_rn(x[i], __dmul_rn((double)D1, q));
        if (!(fabs(rem) <= thr)) {
            q = rint(__ddiv_rn(x[i], (double)D1));
            rem = __dsub_rn(x[i], __dmul_rn((double)D1, q));
        }
        if (!(fabs(q) < 1.0e12)) ok = false;   // also catches NaN
        mi[i] = ok ? (long long)q : 0;
        delta[i] = rem;
    }
    if (!ok) {
        dcrf_flag(status, DCRF_E_NONFINITE);
#pragma unroll
        for (int k = 0; k < D1; ++k) { pslot[a * D1 + k] = -1; pbary[a * D1 + k] = 0.f; }
        return;
    }
    // ranks by delta, descending, ties by index: compared as integers (the
    // FP64 order of finite values, -0 taken as +0), which keeps the 2 (d+1)^2
    // comparisons off the FP64 pipe
    long long dk[D1];
#pragma unroll
    for (int i = 0; i < D1; ++i) {
        const long long bits = __double_as_longlong(delta[i] + 0.0);
        dk[i] = bits < 0 ? bits ^ 0x7fffffffffffffffll : bits;
    }
    int rank[D1];
#pragma unroll
    for (int i = 0; i < D1; ++i) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < D1; ++j)
            r += (dk[j] > dk[i]) || (dk[j] == dk[i] && j < i);
        rank[i] = r;
    }
    long long s = 0;
#pragma unroll
    for (int i = 0; i < D1; ++i) s += mi[i];
    bool moved[D1];
#pragma unroll
    for (int i = 0; i < D1; ++i) moved[i] = false;
    if (s > 0) {
#pragma unroll
        for (int i = 0; i < D1; ++i) {
            if (rank[i] >= D1 - s) { mi[i] -= 1; rank[i] -= (int)(D1 - s); moved[i] = true; }
            else rank[i] += (int)s;
        }
    } else if (s < 0) {
#pragma unroll
        for (int i = 0; i < D1; ++i) {
            if (rank[i] < -s) { mi[i] += 1; rank[i] += (int)(D1 + s); moved[i] = true; }
            else rank[i] += (int)s;
        }
    }
    double ys[D1];
#pragma unroll
    for (int p = 0; p < D1; ++p) ys[p] = 0.0;
#pragma unroll
    for (int i = 0; i < D1; ++i) {
        // the remainder of an unmoved coordinate is the one computed above
        const double dl = moved[i] ? __dsub_rn(x[i], __dmul_rn((double)D1, (double)mi[i])) : delta[i];
#pragma unroll
        for (int p = 0; p < D1; ++p)
            if (rank[i] == p) ys[p] = dl;
    }
    // barycentric weights: differences times RN(1/(d+1)) (within an FP64 ulp
    // of the quotient; the weights are stored as float32)
    double b[D1];
#pragma unroll
    for (int k = 1; k < D1; ++k) b[k] = __dmul_rn(__dsub_rn(ys[D - k], ys[D + 1 - k]), inv);
    b[0] = __dsub_rn(1.0, __dmul_rn(__dsub_rn(ys[0], ys[D]), inv));

    const int64_t base = tab_base[img];
    const uint64_t mask = (uint64_t)tab_mask[img];
#pragma unroll
    for (int k = 0; k < D1; ++k) {
        pbary[a * D1 + k] = (float)b[k];
        long long coord[D];
#pragma unroll
        for (int i = 0; i < D; ++i) coord[i] = D1 * mi[i] + k - (rank[i] >= D1 - k ? D1 : 0);
        uint64_t key;
        int64_t found = -1;
        if (!pack_key<D>(coord, key)) {
            dcrf_flag(status, DCRF_E_KEY_RANGE);
        } else {
            uint64_t h = dcrf_hash64(key);
            const uint64_t probes = max_probe < mask ? max_probe : mask;
            for (uint64_t probe = 0; probe <= probes; ++probe) {
                int64_t slot = base + (int64_t)((h + probe) & mask);
                unsigned long long cur = *((volatile unsigned long long *)&table[slot]);
                if (cur == key) { found = slot; break; }
                if (cur == DCRF_EMPTY_KEY) {
                    unsigned long long prev = atomicCAS(&table[slot], DCRF_EMPTY_KEY, (unsigned long long)key);
                    if (prev == DCRF_EMPTY_KEY || prev == key) { found = slot; break; }
                }
            }
            if (found < 0) dcrf_flag(status, DCRF_E_TABLE_FULL);
        }
        pslot[a * D1 + k] = found;
    }
}

// Vertex numbering by first touch: first[slot] = the lowest incidence index
// a (d+1) + k that lands on the slot.  Vertices are then numbered in that
// order, so pixels that are close in raster order find their corners close
// in memory (and the numbering no longer depends on the hash layout).  The
// first-touch indices of distinct vertices are distinct, so a vertex's number
// is the count of vertices first touched at a lower incidence index: mark the
// first touches, take an exclusive prefix sum over the incidences, and read it
// at each vertex's own first touch.
__global__ void k_first_touch(const int64_t *__restrict__ pslot, int64_t count,
                              unsigned long long *__restrict__ first) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t slot = pslot[i];
    if (slot >= 0 && first[slot] > (unsigned long long)i) atomicMin(first + slot, (unsigned long long)i);
}

__global__ void k_mark_first(const unsigned long long *__restrict__ first, int64_t slots,
                             const int32_t *__restrict__ flag, int32_t *__restrict__ mark) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < slots && flag[i]) mark[first[i]] = 1;
}

__global__ void k_slot_ids(const unsigned long long *__restrict__ first, const int32_t *__restrict__ flag,
                           const int32_t *__restrict__ before, int64_t slots, int32_t *__restrict__ ids) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < slots) ids[i] = flag[i] ? before[first[i]] : 0;
}

__global__ void k_occupied(const unsigned long long *__restrict__ table, int64_t slots,
                           int32_t *__restrict__ flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < slots) flag[i] = table[i] != DCRF_EMPTY_KEY ? 1 : 0;
}

template <int D>
__global__ void k_finalize_slots(const unsigned long long *__restrict__ table, int64_t slots,
                                 const int32_t *__restrict__ scan, const int64_t *__restrict__ tab_base,
                                 int batch, int32_t *__restrict__ keys, int32_t *__restrict__ vimg) {
    constexpr int bits = (64 / D) > 32 ? 32 : (64 / D);
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= slots) return;
    uint64_t key = table[i];
    if (key == DCRF_EMPTY_KEY) return;
    int v = scan[i];
    const long long bias = 1ll << (bits - 1);
    const uint64_t fmask = (bits == 32) ? 0xFFFFFFFFull : ((1ull << bits) - 1);
#pragma unroll
    for (int c = 0; c < D; ++c) keys[(int64_t)v * D + c] = (int32_t)((long long)((key >> (bits * c)) & fmask) - bias);
    vimg[v] = find_image(tab_base, batch, i);
}

__global__ void k_assign_vid(const int64_t *__restrict__ pslot, int64_t count,
                             const int32_t *__restrict__ scan, int32_t *__restrict__ pvid) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) {
        int64_t s = pslot[i];
        pvid[i] = s >= 0 ? scan[s] : -1;
    }
}

__global__ void k_vertex_offsets(const int32_t *__restrict__ scan, const int32_t *__restrict__ flag,
                                 const int64_t *__restrict__ tab_base, int batch, int64_t slots,
                                 int64_t *__restrict__ vert_off) {
    for (int b = threadIdx.x; b < batch; b += blockDim.x) vert_off[b] = scan[tab_base[b]];
    if (threadIdx.x == 0) vert_off[batch] = (int64_t)scan[slots - 1] + flag[slots - 1];
}

template <int D>
__global__ void k_neighbours(const int32_t *__restrict__ keys, const int32_t *__restrict__ vimg, int64_t m,
                             const unsigned long long *__restrict__ table, const int32_t *__restrict__ scan,
                             const int64_t *__restrict__ tab_base, const int64_t *__restrict__ tab_mask,
                             int32_t *__restrict__ nbr) {
    constexpr int D1 = D + 1;
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= m) return;
    long long k0[D];
#pragma unroll
    for (int i = 0; i < D; ++i) k0[i] = keys[v * D + i];
    int img = vimg[v];
    const int64_t base = tab_base[img];
    const uint64_t mask = (uint64_t)tab_mask[img];
    for (int j = 0; j < D1; ++j) {
        for (int side = 0; side < 2; ++side) {
            const long long sgn = side ? 1 : -1;
            long long c[D];
#pragma unroll
            for (int i = 0; i < D; ++i) c[i] = k0[i] + sgn * (i == j ? (long long)D : -1ll);
            int32_t found = -1;
            uint64_t key;
            if (pack_key<D>(c, key)) {
                uint64_t h = dcrf_hash64(key);
                for (uint64_t probe = 0; probe <= mask; ++probe) {
                    int64_t slot = base + (int64_t)((h + probe) & mask);
                    unsigned long long cur = table[slot];
                    if (cur == key) { found = scan[slot]; break; }
                    if (cur == DCRF_EMPTY_KEY) break;
                }
            }
            nbr[(v * D1 + j) * 2 + side] = found;
        }
    }
}

// ---------------------------------------------------------------------------
// filter pieces

__device__ __forceinline__ float4 load4(const float *p, int64_t i) { return reinterpret_cast<const float4 *>(p)[i]; }
__device__ __forceinline__ float4 load4(const __half *p, int64_t i) {
    uint2 raw = reinterpret_cast<const uint2 *>(p)[i];
    __half2 lo = *reinterpret_cast<__half2 *>(&raw.x);
    __half2 hi = *reinterpret_cast<__half2 *>(&raw.y);
    float2 a = __half22float2(lo), b = __half22float2(hi);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store4(float *p, int64_t i, float4 v) { reinterpret_cast<float4 *>(p)[i] = v; }
__device__ __forceinline__ void store4(__half *p, int64_t i, float4 v) {
    __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<uint32_t *>(&lo);
    raw.y = *reinterpret_cast<uint32_t *>(&hi);
    reinterpret_cast<uint2 *>(p)[i] = raw;
}

// One Jacobi pass along axis j: out[v] = in[v]/2 + (in[v - w_j] + in[v + w_j])/4.
template <typename Tin, typename Tout>
__global__ void k_blur_pass(const Tin *__restrict__ in, Tout *__restrict__ out,
                            const int32_t *__restrict__ nbr, int64_t m, int G, int j, int D1) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= m * G) return;
    int64_t v = dcrf_div(idx, G, m * G);
    int g = (int)(idx - v * G);
    int2 nb = reinterpret_cast<const int2 *>(nbr)[v * D1 + j];
    float4 c = load4(in, idx);
    float4 r = make_float4(0.5f * c.x, 0.5f * c.y, 0.5f * c.z, 0.5f * c.w);
    if (nb.x >= 0) {
        float4 q = load4(in, (int64_t)nb.x * G + g);
        r.x += 0.25f * q.x; r.y += 0.25f * q.y; r.z += 0.25f * q.z; r.w += 0.25f * q.w;
    }
    if (nb.y >= 0) {
        float4 q = load4(in, (int64_t)nb.y * G + g);
        r.x += 0.25f * q.x; r.y += 0.25f * q.y; r.z += 0.25f * q.z; r.w += 0.25f * q.w;
    }
    store4(out, idx, r);
}

template <typename T>
static dcrf_status blur_typed(const dcrf_lattice lat, const float *src, T *dst, T *tmp, int Lp,
                              bool reverse, cudaStream_t s) {
    const int D = lat->d, D1 = D + 1, G = Lp / 4;
    const int64_t work = lat->m * G;
    if (work == 0) return DCRF_OK;
    const unsigned nb = blocks_for(work, 256);
    for (int p = 0; p < D1; ++p) {
        int j = reverse ? D - p : p;
        T *out = ((D - p) % 2 == 0) ? dst : tmp;
        ProfScope ps(P_BLUR, s);
        if (p == 0) {
            k_blur_pass<float, T><<<nb, 256, 0, s>>>(src, out, lat->nbr, lat->m, G, j, D1);
        } else {
            T *in = ((D - p + 1) % 2 == 0) ? dst : tmp;
            k_blur_pass<T, T><<<nb, 256, 0, s>>>(in, out, lat->nbr, lat->m, G, j, D1);
        }
        DCRF_LAUNCHED();
    }
    return DCRF_OK;
}

dcrf_status dcrf_blur(const dcrf_lattice lat, const float *src, void *dst, void *tmp, int Lp,
                      int storage, bool reverse, cudaStream_t s) {
    if (storage == DCRF_STORAGE_F16)
        return blur_typed<__half>(lat, src, (__half *)dst, (__half *)tmp, Lp, reverse, s);
    return blur_typed<float>(lat, src, (float *)dst, (float *)tmp, Lp, reverse, s);
}

// S 1 in fixed point: acc[v] += round(2^32 w) over the corners at v (w <= 1,
// so a sum stays far below 2^64); k_ones_rows writes the rows (S 1, 0, 0, 0).
__global__ void k_splat_ones_q(const int32_t *__restrict__ pvid, const float *__restrict__ pbary, int64_t cnt,
                               unsigned long long *acc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const int v = pvid[i];
    if (v >= 0) atomicAdd(acc + v, (unsigned long long)__double2ull_rn(ldexp((double)pbary[i], 32)));
}
__global__ void k_ones_rows(const unsigned long long *__restrict__ acc, int64_t m, float *V,
                            unsigned long long *amax) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const unsigned long long a = v < m ? acc[v] : 0ull;
    if (v < m) reinterpret_cast<float4 *>(V)[v] = make_float4((float)ldexp((double)a, -32), 0.f, 0.f, 0.f);
    const unsigned long long wmax = __reduce_max_sync(0xffffffffu, (unsigned)(a >> 32)) + 1ull;   // upper bound
    if ((threadIdx.x & 31) == 0) atomicMax(amax, wmax);
}

// Dense splat: V[vertex_k(a)][c] += b_k(a) * Y[a][c]; one thread per (point,
// group of four labels), one 16-byte vector reduction per simplex corner.
__global__ void k_splat_dense(const float *__restrict__ Y, int64_t n, int L, int Lp, int D1,
                              const int32_t *__restrict__ pvid, const float *__restrict__ pbary,
                              float *__restrict__ V) {
    const int G = Lp >> 2;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * G) return;
    const int64_t a = dcrf_div(idx, G, n * G);
    const int g = (int)(idx - a * G);
    const int c0 = 4 * g;
    float4 y;
    y.x = c0 + 0 < L ? Y[a * L + c0 + 0] : 0.f;
    y.y = c0 + 1 < L ? Y[a * L + c0 + 1] : 0.f;
    y.z = c0 + 2 < L ? Y[a * L + c0 + 2] : 0.f;
    y.w = c0 + 3 < L ? Y[a * L + c0 + 3] : 0.f;
    for (int k = 0; k < D1; ++k) {
        const int v = pvid[a * D1 + k];
        if (v < 0) continue;
        const float w = pbary[a * D1 + k];
        atomicAdd(reinterpret_cast<float4 *>(V + (int64_t)v * Lp + c0), make_float4(w * y.x, w * y.y, w * y.z, w * y.w));
    }
}

dcrf_status dcrf_splat_dense(const dcrf_lattice lat, const float *Y, int L, float *V, int Lp,
                             cudaStream_t s) {
    if (lat->n == 0) return DCRF_OK;
    ProfScope ps(P_SPLAT_DENSE, s);
    k_splat_dense<<<blocks_for(lat->n * (Lp / 4), 256), 256, 0, s>>>(Y, lat->n, L, Lp, lat->d + 1, lat->pvid,
                                                                   lat->pbary, V);
    DCRF_LAUNCHED();
    return DCRF_OK;
}

// Slice: out[a][c] = s0 * sum_k b_k(a) V[vertex_k(a)][c].
template <typename T>
__global__ void k_slice(const T *__restrict__ V, int64_t n, int L, int G, int D1,
                        const int32_t *__restrict__ pvid, const float *__restrict__ pbary, float s0,
                        float *__restrict__ out) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * G) return;
    int64_t a = dcrf_div(idx, G, n * G);
    int g = (int)(idx - a * G);
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < D1; ++k) {
        int v = pvid[a * D1 + k];
        if (v < 0) continue;
        float w = pbary[a * D1 + k];
        float4 q = load4(V, (int64_t)v * G + g);
        r.x += w * q.x; r.y += w * q.y; r.z += w * q.z; r.w += w * q.w;
    }
    float vals[4] = {r.x, r.y, r.z, r.w};
    for (int i = 0; i < 4; ++i) {
        int c = 4 * g + i;
        if (c < L) out[a * L + c] = s0 * vals[i];
    }
}

dcrf_status dcrf_slice(const dcrf_lattice lat, const void *V, int Lp, int L, int storage, float *out,
                       cudaStream_t s) {
    if (lat->n == 0) return DCRF_OK;
    const int G = Lp / 4;
    const unsigned nb = blocks_for(lat->n * G, 256);
    ProfScope ps(P_SLICE, s);
    if (storage == DCRF_STORAGE_F16)
        k_slice<__half><<<nb, 256, 0, s>>>((const __half *)V, lat->n, L, G, lat->d + 1, lat->pvid, lat->pbary,
                                           (float)lat->s0, out);
    else
        k_slice<float><<<nb, 256, 0, s>>>((const float *)V, lat->n, L, G, lat->d + 1, lat->pvid, lat->pbary,
                                          (float)lat->s0, out);
    DCRF_LAUNCHED();
    return DCRF_OK;
}

dcrf_status dcrf_slice_f32(const dcrf_lattice lat, const float *V, int Lp, int L, float *out, cudaStream_t s) {
    return dcrf_slice(lat, V, Lp, L, DCRF_STORAGE_F32, out, s);
}

static dcrf_status filter_impl(const dcrf_lattice lat, const float *Y, int L, float *out, int storage,
                               bool reverse, cudaStream_t s) {
    if (!lat || !Y || !out || L < 1 || L > DCRF_MAX_L) return DCRF_E_INVAL;
    if (storage != DCRF_STORAGE_F32 && storage != DCRF_STORAGE_F16) return DCRF_E_INVAL;
    if (lat->n == 0) return DCRF_OK;
    const int Lp = dcrf_round4(L);
    const size_t esz = storage == DCRF_STORAGE_F16 ? 2 : 4;
    Scratch sc(s);
    float *V;
    char *dst, *tmp;
    DCRF_CHECK_STATUS(sc.get(&V, (size_t)lat->m * Lp));
    DCRF_CHECK_STATUS(sc.get(&dst, (size_t)lat->m * Lp * esz));
    DCRF_CHECK_STATUS(sc.get(&tmp, (size_t)lat->m * Lp * esz));
    DCRF_TRY(cudaMemsetAsync(V, 0, (size_t)lat->m * Lp * sizeof(float), s));
    DCRF_CHECK_STATUS(dcrf_splat_dense(lat, Y, L, V, Lp, s));
    DCRF_CHECK_STATUS(dcrf_blur(lat, V, dst, tmp, Lp, storage, reverse, s));
    return dcrf_slice(lat, dst, Lp, L, storage, out, s);
}

extern "C" dcrf_status dcrf_filter(dcrf_lattice lat, const float *Y, int L, float *out, int storage,
                                   dcrf_stream stream) {
    if (Y == out) return DCRF_E_INVAL;
    return filter_impl(lat, Y, L, out, storage, false, (cudaStream_t)stream);
}

extern "C" dcrf_status dcrf_filter_adjoint(dcrf_lattice lat, const float *U, int L, float *out,
                                           int storage, dcrf_stream stream) {
    if (U == out) return DCRF_E_INVAL;
    return filter_impl(lat, U, L, out, storage, true, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// build driver

// The lattice's arrays come from the library's stream-ordered pool of its
// device (a build maps no new memory once the pool holds enough, and a destroy
// unmaps none).  They are freed on that device's legacy default stream once
// no work that may read them is left (callers synchronise first).
template <typename T>
static dcrf_status lattice_alloc(T **p, size_t count, cudaStream_t s) {
    return dcrf_alloc(p, count > 0 ? count : 1, s);
}

static void lattice_free(dcrf_lattice lat) {
    if (!lat) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (lat->device >= 0 && lat->device != cur) cudaSetDevice(lat->device);
    void *arrays[] = {lat->point_off_d, lat->vert_off_d, lat->pvid, lat->pbary, lat->keys,
                      lat->nbr,         lat->vimg,       lat->ones, lat->status};
    for (void *p : arrays)
        if (p) cudaFreeAsync(p, 0);
    if (lat->device >= 0 && lat->device != cur) cudaSetDevice(cur);
    delete lat;
}

__global__ void k_fill(float *p, float v, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

dcrf_status dcrf_fill(float *p, float v, int64_t n, cudaStream_t s) {
    if (n <= 0) return DCRF_OK;
    k_fill<<<blocks_for(n, 256), 256, 0, s>>>(p, v, n);
    DCRF_LAUNCHED();
    return DCRF_OK;
}

template <int D>
static dcrf_status build_typed(dcrf_lattice lat, const float *feat, cudaStream_t s) {
    constexpr int D1 = D + 1;
    const int batch = lat->batch;
    const int64_t n = lat->n;
    EmbedParams P;
    const double alpha = (double)D1 * std::sqrt(2.0 / 3.0);
    for (int j = 0; j < DCRF_MAX_D; ++j)
        P.sig[j] = j < D ? alpha / std::sqrt((double)((j + 1) * (j + 2))) : 0.0;
    P.batch = batch;
    lat->s0 = std::pow(2.0 * M_PI, D / 2.0) * std::pow(alpha, (double)D) / std::pow((double)D1, D - 0.5);

    // testing hook: DCRF_TABLE_SLOTS caps every segment (power of two), so that
    // the bounded probing and its DCRF_E_TABLE_FULL report can be exercised
    int64_t cap_limit = 0;
    if (const char *lim = std::getenv("DCRF_TABLE_SLOTS")) cap_limit = std::atoll(lim);

    Scratch sc(s);
    unsigned long long *table = nullptr;
    int64_t *pslot, *base_d, *mask_d;
    int32_t *flag = nullptr, *scan = nullptr;
    DCRF_CHECK_STATUS(sc.get(&pslot, (size_t)n * D1 + 1));
    DCRF_CHECK_STATUS(sc.get(&base_d, batch));
    DCRF_CHECK_STATUS(sc.get(&mask_d, batch));
    int64_t slots = 0;
    // One power-of-two table segment per image.  Vertices are far fewer than
    // the n_b (d+1) corners (neighbouring points share them), so the first
    // attempt sizes a segment for n_b (d+1) / 8 vertices at load <= 1/2; if a
    // segment fills up (bounded probing reports DCRF_E_TABLE_FULL) the build
    // runs again with room for every corner.  The table is the largest buffer
    // of the build, so the first attempt is the cheap one.
    for (int attempt = 0; attempt < 2; ++attempt) {
        std::vector<int64_t> base(batch), mask(batch);
        slots = 0;
        for (int b = 0; b < batch; ++b) {
            const int64_t nb = lat->point_off[b + 1] - lat->point_off[b];
            const int64_t corners = nb * D1;
            int64_t want = attempt == 0 ? corners / 4 : 2 * corners;
            if (want < 64) want = 64;
            int64_t cap = 64;
            while (cap < want) cap <<= 1;
            if (cap_limit >= 1) {
                int64_t c2 = 1;
                while (c2 * 2 <= cap_limit) c2 <<= 1;
                cap = std::min(cap, c2);
            }
            base[b] = slots;
            mask[b] = cap - 1;
            slots += cap;
        }
        if (slots >= (1ll << 31)) return DCRF_E_INVAL;   // vertex ids are int32
        DCRF_CHECK_STATUS(sc.get(&table, slots));
        DCRF_CHECK_STATUS(sc.get(&flag, slots));
        DCRF_CHECK_STATUS(sc.get(&scan, slots));
        DCRF_TRY(cudaMemcpyAsync(base_d, base.data(), batch * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        DCRF_TRY(cudaMemcpyAsync(mask_d, mask.data(), batch * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        DCRF_TRY(cudaMemsetAsync(table, 0xFF, slots * sizeof(unsigned long long), s));
        DCRF_TRY(cudaMemsetAsync(lat->status, 0, sizeof(int), s));
        if (n > 0) {
            ProfScope ps(P_EMBED, s);
            // the first attempt gives up after 256 probes (a crowded table
            // then costs little before the second attempt)
            k_embed_insert<D><<<blocks_for(n, 128), 128, 0, s>>>(feat, n, P, lat->point_off_d, base_d, mask_d,
                                                                 table, pslot, lat->pbary, lat->status,
                                                                 attempt == 0 ? 255ull : ~0ull);
            DCRF_LAUNCHED();
        }
        int hstatus = 0;
        DCRF_TRY(cudaMemcpyAsync(&hstatus, lat->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DCRF_TRY(cudaStreamSynchronize(s));
        if (hstatus == DCRF_E_TABLE_FULL && attempt == 0) continue;
        if (hstatus != 0) return (dcrf_status)hstatus;
        break;
    }
    k_occupied<<<blocks_for(slots, 256), 256, 0, s>>>(table, slots, flag);
    DCRF_LAUNCHED();
    DCRF_CHECK_STATUS(dcrf_scan(flag, scan, slots, false, s));
    k_vertex_offsets<<<1, 1024, 0, s>>>(scan, flag, base_d, batch, slots, lat->vert_off_d);
    DCRF_LAUNCHED();
    lat->vert_off.assign(batch + 1, 0);
    DCRF_TRY(cudaMemcpyAsync(lat->vert_off.data(), lat->vert_off_d, (batch + 1) * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
    DCRF_TRY(cudaStreamSynchronize(s));
    lat->m = lat->vert_off[batch];
    const int64_t m = lat->m;

    // renumber the vertices by first touch (image ranges are unchanged: every
    // vertex of image b is first touched by a point of image b)
    int32_t *ids = scan;
    if (m > 1) {
        unsigned long long *first;
        int32_t *mark, *before;
        DCRF_CHECK_STATUS(sc.get(&first, slots));
        DCRF_CHECK_STATUS(sc.get(&mark, (size_t)n * D1));
        DCRF_CHECK_STATUS(sc.get(&before, (size_t)n * D1));
        DCRF_CHECK_STATUS(sc.get(&ids, slots));
        DCRF_TRY(cudaMemsetAsync(first, 0xFF, slots * sizeof(unsigned long long), s));
        DCRF_TRY(cudaMemsetAsync(mark, 0, (size_t)n * D1 * sizeof(int32_t), s));
        k_first_touch<<<blocks_for(n * D1, 256), 256, 0, s>>>(pslot, n * D1, first);
        DCRF_LAUNCHED();
        k_mark_first<<<blocks_for(slots, 256), 256, 0, s>>>(first, slots, flag, mark);
        DCRF_LAUNCHED();
        DCRF_CHECK_STATUS(dcrf_scan(mark, before, n * D1, false, s));
        k_slot_ids<<<blocks_for(slots, 256), 256, 0, s>>>(first, flag, before, slots, ids);
        DCRF_LAUNCHED();
    }

    DCRF_CHECK_STATUS(lattice_alloc(&lat->keys, (size_t)m * D, s));
    DCRF_CHECK_STATUS(lattice_alloc(&lat->vimg, (size_t)m, s));
    DCRF_CHECK_STATUS(lattice_alloc(&lat->nbr, (size_t)m * D1 * 2, s));
    k_finalize_slots<D><<<blocks_for(slots, 256), 256, 0, s>>>(table, slots, ids, base_d, batch, lat->keys,
                                                               lat->vimg);
    DCRF_LAUNCHED();
    if (n > 0) {
        k_assign_vid<<<blocks_for(n * D1, 256), 256, 0, s>>>(pslot, n * D1, ids, lat->pvid);
        DCRF_LAUNCHED();
    }
    if (m > 0) {
        k_neighbours<D><<<blocks_for(m, 128), 128, 0, s>>>(lat->keys, lat->vimg, m, table, ids, base_d, mask_d,
                                                           lat->nbr);
        DCRF_LAUNCHED();
    }
    unsigned long long s1bound = 0;
    // K~ 1 for the d vector of Eq. 11; S 1 is summed in 64-bit fixed point
    // (integer sums: the same lattice comes out of every build of the same
    // points, bit for bit)
    if (n > 0 && m > 0) {
        float *V, *A, *B;
        unsigned long long *acc;
        DCRF_CHECK_STATUS(sc.get(&V, (size_t)m * 4));
        DCRF_CHECK_STATUS(sc.get(&A, (size_t)m * 4));
        DCRF_CHECK_STATUS(sc.get(&B, (size_t)m * 4));
        DCRF_CHECK_STATUS(sc.get(&acc, (size_t)m + 1));
        DCRF_TRY(cudaMemsetAsync(acc, 0, (size_t)(m + 1) * sizeof(unsigned long long), s));
        k_splat_ones_q<<<blocks_for(n * D1, 256), 256, 0, s>>>(lat->pvid, lat->pbary, n * D1, acc);
        DCRF_LAUNCHED();
        // acc[m]: an integer upper bound of max_v (S 1)_v (read at the sync below)
        k_ones_rows<<<blocks_for(m, 256), 256, 0, s>>>(acc, m, V, acc + m);
        DCRF_LAUNCHED();
        DCRF_TRY(cudaMemcpyAsync(&s1bound, acc + m, sizeof(s1bound), cudaMemcpyDeviceToHost, s));
        DCRF_CHECK_STATUS(dcrf_blur(lat, V, A, B, 4, DCRF_STORAGE_F32, false, s));
        k_slice<float><<<blocks_for(n, 256), 256, 0, s>>>(A, n, 1, 1, D1, lat->pvid, lat->pbary, (float)lat->s0,
                                                          lat->ones);
        DCRF_LAUNCHED();
    }
    int hstatus = 0;
    DCRF_TRY(cudaMemcpyAsync(&hstatus, lat->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    DCRF_TRY(cudaStreamSynchronize(s));
    if (hstatus != 0) return (dcrf_status)hstatus;
    lat->s1max = (double)s1bound;
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_lattice_build_batch(const float *features, const int64_t *offsets, int batch,
                                                int d, dcrf_stream stream, dcrf_lattice *out) {
    if (!out) return DCRF_E_INVAL;
    *out = nullptr;
    if (!offsets || batch < 1 || d < 1 || d > DCRF_MAX_D) return DCRF_E_INVAL;
    if (offsets[0] != 0) return DCRF_E_INVAL;
    for (int b = 0; b < batch; ++b)
        if (offsets[b + 1] < offsets[b]) return DCRF_E_INVAL;
    const int64_t n = offsets[batch];
    if (n > 0 && !features) return DCRF_E_INVAL;
    if (n >= (1ll << 31) / (d + 1)) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    dcrf_lattice lat = new (std::nothrow) dcrf_lattice_s();
    if (!lat) return DCRF_E_NOMEM;
    lat->d = d;
    lat->n = n;
    lat->batch = batch;
    lat->point_off.assign(offsets, offsets + batch + 1);
    const int D1 = d + 1;
    if (cudaStreamGetDevice(s, &lat->device) != cudaSuccess) { delete lat; return DCRF_E_CUDA; }
    dcrf_status ast = DCRF_OK;
    if (ast == DCRF_OK) ast = lattice_alloc(&lat->point_off_d, (size_t)batch + 1, s);
    if (ast == DCRF_OK) ast = lattice_alloc(&lat->vert_off_d, (size_t)batch + 1, s);
    if (ast == DCRF_OK) ast = lattice_alloc(&lat->pvid, (size_t)n * D1, s);
    if (ast == DCRF_OK) ast = lattice_alloc(&lat->pbary, (size_t)n * D1, s);
    if (ast == DCRF_OK) ast = lattice_alloc(&lat->ones, (size_t)n, s);
    if (ast == DCRF_OK) ast = lattice_alloc(&lat->status, 1, s);
    if (ast != DCRF_OK) { cudaStreamSynchronize(s); lattice_free(lat); return ast; }
    cudaError_t e = cudaMemcpyAsync(lat->point_off_d, offsets, (batch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(lat->status, 0, sizeof(int), s);
    if (e != cudaSuccess) { cudaStreamSynchronize(s); lattice_free(lat); return DCRF_E_CUDA; }
    dcrf_status st;
    switch (d) {
    case 1: st = build_typed<1>(lat, features, s); break;
    case 2: st = build_typed<2>(lat, features, s); break;
    case 3: st = build_typed<3>(lat, features, s); break;
    case 4: st = build_typed<4>(lat, features, s); break;
    case 5: st = build_typed<5>(lat, features, s); break;
    case 6: st = build_typed<6>(lat, features, s); break;
    case 7: st = build_typed<7>(lat, features, s); break;
    default: st = build_typed<8>(lat, features, s); break;
    }
    if (st != DCRF_OK) {
        cudaStreamSynchronize(s);
        lattice_free(lat);
        return st;
    }
    // dcrf_filter_static's scratch address for this device, looked up here
    // (outside any capture: the build synchronises) so that its calls find it
    unsigned char *scratch = nullptr;
    (void)dcrf_static_scratch(s, &scratch);
    *out = lat;
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_lattice_build(const float *features, int64_t n, int d, dcrf_stream stream,
                                          dcrf_lattice *out) {
    int64_t off[2] = {0, n};
    if (n < 0) return DCRF_E_INVAL;
    return dcrf_lattice_build_batch(features, off, 1, d, stream, out);
}

extern "C" dcrf_status dcrf_lattice_destroy(dcrf_lattice lat) {
    if (!lat) return DCRF_E_INVAL;
    cudaDeviceSynchronize();
    lattice_free(lat);
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_lattice_info(dcrf_lattice lat, int64_t *n, int *d, int64_t *m, int *batch) {
    if (!lat) return DCRF_E_INVAL;
    if (n) *n = lat->n;
    if (d) *d = lat->d;
    if (m) *m = lat->m;
    if (batch) *batch = lat->batch;
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_lattice_vertex_offsets(dcrf_lattice lat, int64_t *offsets) {
    if (!lat || !offsets) return DCRF_E_INVAL;
    for (int b = 0; b <= lat->batch; ++b) offsets[b] = lat->vert_off[b];
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_lattice_status(dcrf_lattice lat, dcrf_stream stream) {
    if (!lat) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    DCRF_TRY(cudaMemcpyAsync(&h, lat->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    DCRF_TRY(cudaMemsetAsync(lat->status, 0, sizeof(int), s));
    DCRF_TRY(cudaStreamSynchronize(s));
    return (dcrf_status)h;
}

// ---------------------------------------------------------------------------
// check mode: the tables the kernels index with

__device__ __forceinline__ int image_of(const int64_t *off, int batch, int64_t i) {
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// every corner's vertex is -1 or one of its image's vertices; weights are
// finite, in [0, 1] and sum to one (1e-5)
__global__ void k_check_points(const int32_t *__restrict__ pvid, const float *__restrict__ pbary, int64_t n, int d1,
                               const int64_t *__restrict__ poff, const int64_t *__restrict__ voff, int batch,
                               unsigned long long *bad) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int b = image_of(poff, batch, a);
    float sum = 0.f;
    int errs = 0;
    for (int k = 0; k < d1; ++k) {
        const int v = pvid[a * d1 + k];
        const float w = pbary[a * d1 + k];
        if (v != -1 && (v < voff[b] || v >= voff[b + 1])) ++errs;
        if (!(w >= -1e-6f && w <= 1.f + 1e-6f)) ++errs;
        sum += w;
    }
    if (!(fabsf(sum - 1.f) <= 1e-5f)) ++errs;
    if (errs) atomicAdd(bad, (unsigned long long)errs);
}

// every blur neighbour is -1 or a vertex of the same image
__global__ void k_check_neighbours(const int32_t *__restrict__ nbr, int64_t m, int d1, const int64_t *__restrict__ voff,
                                   int batch, unsigned long long *bad) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= m) return;
    const int b = image_of(voff, batch, v);
    int errs = 0;
    for (int j = 0; j < 2 * d1; ++j) {
        const int u = nbr[v * 2 * d1 + j];
        if (u != -1 && (u < voff[b] || u >= voff[b + 1])) ++errs;
    }
    if (errs) atomicAdd(bad, (unsigned long long)errs);
}

extern "C" dcrf_status dcrf_check_lattice_tables(const int32_t *point_vertex, const float *point_weight, int64_t n,
                                                 int d, const int32_t *neighbours, int64_t m,
                                                 const int64_t *point_offsets, const int64_t *vertex_offsets,
                                                 int batch, int64_t *bad_entries, dcrf_stream stream) {
    if (bad_entries) *bad_entries = 0;
    if (d < 1 || d > DCRF_MAX_D || n < 0 || m < 0 || batch < 1 || !point_offsets || !vertex_offsets)
        return DCRF_E_INVAL;
    if ((n > 0 && (!point_vertex || !point_weight)) || (m > 0 && !neighbours)) return DCRF_E_INVAL;
    if (point_offsets[0] != 0 || point_offsets[batch] != n || vertex_offsets[0] != 0 || vertex_offsets[batch] != m)
        return DCRF_E_INVAL;
    for (int b = 0; b < batch; ++b)
        if (point_offsets[b + 1] < point_offsets[b] || vertex_offsets[b + 1] < vertex_offsets[b]) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    int64_t *poff, *voff;
    unsigned long long *bad;
    DCRF_CHECK_STATUS(sc.get(&poff, (size_t)batch + 1));
    DCRF_CHECK_STATUS(sc.get(&voff, (size_t)batch + 1));
    DCRF_CHECK_STATUS(sc.get(&bad, 1));
    DCRF_TRY(cudaMemcpyAsync(poff, point_offsets, (batch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DCRF_TRY(cudaMemcpyAsync(voff, vertex_offsets, (batch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DCRF_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
    if (n > 0) {
        k_check_points<<<blocks_for(n, 256), 256, 0, s>>>(point_vertex, point_weight, n, d + 1, poff, voff, batch, bad);
        DCRF_LAUNCHED();
    }
    if (m > 0) {
        k_check_neighbours<<<blocks_for(m, 256), 256, 0, s>>>(neighbours, m, d + 1, voff, batch, bad);
        DCRF_LAUNCHED();
    }
    unsigned long long h = 0;
    DCRF_TRY(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s));
    DCRF_TRY(cudaStreamSynchronize(s));
    if (bad_entries) *bad_entries = (int64_t)h;
    return h ? DCRF_E_INVAL : DCRF_OK;
}

extern "C" dcrf_status dcrf_lattice_validate(dcrf_lattice lat, int64_t *bad_entries, dcrf_stream stream) {
    if (!lat) return DCRF_E_INVAL;
    return dcrf_check_lattice_tables(lat->pvid, lat->pbary, lat->n, lat->d, lat->nbr, lat->m, lat->point_off.data(),
                                     lat->vert_off.data(), lat->batch, bad_entries, stream);
}

extern "C" dcrf_status dcrf_lattice_export(dcrf_lattice lat, int32_t *keys, int32_t *point_vertex,
                                           float *point_weight, int32_t *neighbours, dcrf_stream stream) {
    if (!lat) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int D1 = lat->d + 1;
    if (keys && lat->m)
        DCRF_TRY(cudaMemcpyAsync(keys, lat->keys, lat->m * lat->d * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (point_vertex && lat->n)
        DCRF_TRY(cudaMemcpyAsync(point_vertex, lat->pvid, lat->n * D1 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (point_weight && lat->n)
        DCRF_TRY(cudaMemcpyAsync(point_weight, lat->pbary, lat->n * D1 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (neighbours && lat->m)
        DCRF_TRY(cudaMemcpyAsync(neighbours, lat->nbr, lat->m * D1 * 2 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    return DCRF_OK;
}
