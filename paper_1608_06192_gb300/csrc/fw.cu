// Frank-Wolfe on the convex QP relaxation and CCCP on the generic DC relaxation.
//
// Algorithm 1 with the closed-form step and the product reuse of Appendix B,
// and Algorithm 2 (Section 5.1).  The operator is Psi + D with
// Psi = mu (x) (K~ - sum_w I) (Eq. 7) and d_a(i) = sum_j |mu_ij| c_a (Eq. 11),
// K~ = sum_m w_m s0_m S_m^T B_m S_m (one permutohedral lattice per kernel).
//
// Product reuse is done on the lattice instead of the pixels: since
// y^{t+1} = y^t + alpha (s - y^t) and splat/blur are linear, the solver keeps
//   Ylat = S y   and   BY = B S y          (per lattice, [M][Lp] float32)
// and updates them with the same convex combination, so (Psi + D) y^{t+1} is
// one slice of (1 - alpha) BY + alpha BS per pixel.  The one filter of every
// iteration is the splat and blur of the one-hot s; the line-search terms
// <y, P_s> and <s, P_s> use S^T = slice: <u, K~ v> = sum_m w_m s0_m <S u, B S v>
// is a dot product over lattice vertices.  Each iteration therefore reads the
// per-pixel state (y, phi - d, s, simplex table) once and writes y and s once.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <cstring>

#include "common.cuh"

#include "fw_pixel.cuh"

namespace {

// Blur pass `p` of every lattice in one launch (lattice m takes part while
// p < d_m + 1): out[v] = in[v]/2 + (in[v - w_p] + in[v + w_p])/4 on whole rows
// of LP labels, one thread per vertex.  Pass 0 reads the fixed-point splat Sq;
// the last pass of lattice m lands in BS, earlier ones alternate with tmp.
template <typename T>
__device__ __forceinline__ void row_load(const T *p, int64_t v, int LP, int q, float (&o)[8]);
template <>
__device__ __forceinline__ void row_load<float>(const float *p, int64_t v, int LP, int q, float (&o)[8]) {
    const float4 *r = reinterpret_cast<const float4 *>(p + v * LP + 8 * q);
    const float4 a = r[0], b = r[1];
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
template <>
__device__ __forceinline__ void row_load<__half>(const __half *p, int64_t v, int LP, int q, float (&o)[8]) {
    const uint4 raw = *reinterpret_cast<const uint4 *>(p + v * LP + 8 * q);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
    const float2 c = __half22float2(*reinterpret_cast<const __half2 *>(&raw.z));
    const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&raw.w));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y; o[4] = c.x; o[5] = c.y; o[6] = d.x; o[7] = d.y;
}
// Eight labels of a fixed-point splat row, as values: u * inv (inv = 2^-k).
__device__ __forceinline__ void row_load_q(const uint32_t *p, int64_t v, int LP, int q, float inv, float (&o)[8]) {
    const uint4 *r = reinterpret_cast<const uint4 *>(p + v * LP + 8 * q);
    const uint4 a = r[0], b = r[1];
    o[0] = (float)a.x * inv; o[1] = (float)a.y * inv; o[2] = (float)a.z * inv; o[3] = (float)a.w * inv;
    o[4] = (float)b.x * inv; o[5] = (float)b.y * inv; o[6] = (float)b.z * inv; o[7] = (float)b.w * inv;
}
__device__ __forceinline__ void row_store(float *p, int64_t v, int LP, int q, const float (&o)[8]) {
    float4 *r = reinterpret_cast<float4 *>(p + v * LP + 8 * q);
    r[0] = make_float4(o[0], o[1], o[2], o[3]);
    r[1] = make_float4(o[4], o[5], o[6], o[7]);
}
__device__ __forceinline__ void row_store(__half *p, int64_t v, int LP, int q, const float (&o)[8]) {
    __half2 h0 = __floats2half2_rn(o[0], o[1]), h1 = __floats2half2_rn(o[2], o[3]);
    __half2 h2 = __floats2half2_rn(o[4], o[5]), h3 = __floats2half2_rn(o[6], o[7]);
    uint4 raw;
    raw.x = *reinterpret_cast<uint32_t *>(&h0);
    raw.y = *reinterpret_cast<uint32_t *>(&h1);
    raw.z = *reinterpret_cast<uint32_t *>(&h2);
    raw.w = *reinterpret_cast<uint32_t *>(&h3);
    *reinterpret_cast<uint4 *>(p + v * LP + 8 * q) = raw;
}

struct BlurLat {
    const int32_t *nbr;
    const uint32_t *src0;   // Sq (fixed point) for pass 0
    const float *qs;        // its scales {2^k, 2^-k}
    void *dst;           // BS
    void *tmp;
    int64_t m;
    int d1;
};
struct BlurSet {
    BlurLat l[DCRF_MAX_KERNELS];
    int64_t start[DCRF_MAX_KERNELS + 1];   // prefix of the vertex counts that take part
    int nk;
};

template <int LP, typename T>
__global__ void __launch_bounds__(256) k_fw_blur(BlurSet B, int p) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int mm = 0;
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k < B.nk && g >= B.start[k]) mm = k;
    if (g >= B.start[B.nk]) return;
    BlurLat lt = B.l[0];
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k == mm) lt = B.l[k];
    if (p >= lt.d1) return;
    const int64_t v = g - B.start[mm];
    const int D = lt.d1 - 1;
    T *out = ((D - p) % 2 == 0) ? (T *)lt.dst : (T *)lt.tmp;
    const int2 nb = reinterpret_cast<const int2 *>(lt.nbr)[v * lt.d1 + p];
    if constexpr (sizeof(T) == 2 && LP <= 24) {
        if (p > 0) {
            // half rows: every 16-byte load of the three rows is issued before
            // any arithmetic or store (the output is never an input, but the
            // compiler cannot know that); raw halves keep the registers low
            const uint4 *in = reinterpret_cast<const uint4 *>(((D - p + 1) % 2 == 0) ? lt.dst : lt.tmp);
            uint4 c[LP / 8], a[LP / 8], b[LP / 8];
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int q = 0; q < LP / 8; ++q) {
                c[q] = in[v * (LP / 8) + q];
                a[q] = nb.x >= 0 ? in[(int64_t)nb.x * (LP / 8) + q] : z;
                b[q] = nb.y >= 0 ? in[(int64_t)nb.y * (LP / 8) + q] : z;
            }
#pragma unroll
            for (int q = 0; q < LP / 8; ++q) {
                const __half2 *hc = reinterpret_cast<const __half2 *>(&c[q]);
                const __half2 *ha = reinterpret_cast<const __half2 *>(&a[q]);
                const __half2 *hb = reinterpret_cast<const __half2 *>(&b[q]);
                float o[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 fc = __half22float2(hc[j]), fa = __half22float2(ha[j]), fb = __half22float2(hb[j]);
                    o[2 * j] = 0.5f * fc.x + 0.25f * fa.x + 0.25f * fb.x;
                    o[2 * j + 1] = 0.5f * fc.y + 0.25f * fa.y + 0.25f * fb.y;
                }
                row_store(out, v, LP, q, o);
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < LP / 8; ++q) {
        float c[8], a[8], b[8];
        if (p == 0) {
            const float inv = __ldg(lt.qs + 1);
            row_load_q(lt.src0, v, LP, q, inv, c);
            if (nb.x >= 0) row_load_q(lt.src0, nb.x, LP, q, inv, a);
            if (nb.y >= 0) row_load_q(lt.src0, nb.y, LP, q, inv, b);
        } else {
            const T *in = ((D - p + 1) % 2 == 0) ? (const T *)lt.dst : (const T *)lt.tmp;
            row_load<T>(in, v, LP, q, c);
            if (nb.x >= 0) row_load<T>(in, nb.x, LP, q, a);
            if (nb.y >= 0) row_load<T>(in, nb.y, LP, q, b);
        }
        float o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            o[j] = 0.5f * c[j] + (nb.x >= 0 ? 0.25f * a[j] : 0.f) + (nb.y >= 0 ? 0.25f * b[j] : 0.f);
        row_store(out, v, LP, q, o);
    }
}

// Persistent blur pass: a grid of resident blocks strides over the vertex
// rows, and every thread loads the neighbour pair of its next row while it
// works on the current one, so a row waits for one round trip to memory
// (its three rows) instead of two (the pair, then the rows).  Same
// arithmetic as k_fw_blur.
template <int LP, typename T>
__device__ __forceinline__ bool blur2_locate(const BlurSet &B, int p, int64_t g, BlurLat &lt, int64_t &v) {
    int mm = 0;
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k < B.nk && g >= B.start[k]) mm = k;
    lt = B.l[0];
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k == mm) lt = B.l[k];
    v = g - B.start[mm];
    return p < lt.d1;
}

template <int LP, typename T>
__global__ void __launch_bounds__(256) k_fw_blur2(BlurSet B, int p, int64_t work) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    BlurLat lt;
    int64_t v = 0;
    bool live = g < work && blur2_locate<LP, T>(B, p, g, lt, v);
    int2 nb = live ? reinterpret_cast<const int2 *>(lt.nbr)[v * lt.d1 + p] : make_int2(-1, -1);
    while (g < work) {
        // the next row's lattice, vertex and neighbour pair, in flight during this row
        const int64_t gn = g + stride;
        BlurLat ln;
        int64_t vn = 0;
        const bool live_n = gn < work && blur2_locate<LP, T>(B, p, gn, ln, vn);
        const int2 nbn = live_n ? reinterpret_cast<const int2 *>(ln.nbr)[vn * ln.d1 + p] : make_int2(-1, -1);
        if (live) {
            const int D = lt.d1 - 1;
            T *out = ((D - p) % 2 == 0) ? (T *)lt.dst : (T *)lt.tmp;
            bool done = false;
            if constexpr (sizeof(T) == 2 && LP <= 24) {
                if (p > 0) {
                    const uint4 *in = reinterpret_cast<const uint4 *>(((D - p + 1) % 2 == 0) ? lt.dst : lt.tmp);
                    uint4 c[LP / 8], a[LP / 8], b[LP / 8];
                    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                    for (int q = 0; q < LP / 8; ++q) {
                        c[q] = in[v * (LP / 8) + q];
                        a[q] = nb.x >= 0 ? in[(int64_t)nb.x * (LP / 8) + q] : z;
                        b[q] = nb.y >= 0 ? in[(int64_t)nb.y * (LP / 8) + q] : z;
                    }
#pragma unroll
                    for (int q = 0; q < LP / 8; ++q) {
                        const __half2 *hc = reinterpret_cast<const __half2 *>(&c[q]);
                        const __half2 *ha = reinterpret_cast<const __half2 *>(&a[q]);
                        const __half2 *hb = reinterpret_cast<const __half2 *>(&b[q]);
                        float o[8];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float2 fc = __half22float2(hc[j]), fa = __half22float2(ha[j]);
                            const float2 fb = __half22float2(hb[j]);
                            o[2 * j] = 0.5f * fc.x + 0.25f * fa.x + 0.25f * fb.x;
                            o[2 * j + 1] = 0.5f * fc.y + 0.25f * fa.y + 0.25f * fb.y;
                        }
                        row_store(out, v, LP, q, o);
                    }
                    done = true;
                }
            }
            if (!done) {
#pragma unroll
                for (int q = 0; q < LP / 8; ++q) {
                    float c[8], a[8], b[8];
                    if (p == 0) {
                        const float inv = __ldg(lt.qs + 1);
                        row_load_q(lt.src0, v, LP, q, inv, c);
                        if (nb.x >= 0) row_load_q(lt.src0, nb.x, LP, q, inv, a);
                        if (nb.y >= 0) row_load_q(lt.src0, nb.y, LP, q, inv, b);
                    } else {
                        const T *in = ((D - p + 1) % 2 == 0) ? (const T *)lt.dst : (const T *)lt.tmp;
                        row_load<T>(in, v, LP, q, c);
                        if (nb.x >= 0) row_load<T>(in, nb.x, LP, q, a);
                        if (nb.y >= 0) row_load<T>(in, nb.y, LP, q, b);
                    }
                    float o[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        o[j] = 0.5f * c[j] + (nb.x >= 0 ? 0.25f * a[j] : 0.f) + (nb.y >= 0 ? 0.25f * b[j] : 0.f);
                    row_store(out, v, LP, q, o);
                }
            }
        }
        g = gn;
        lt = ln;
        v = vn;
        live = live_n;
        nb = nbn;
    }
}

// Label-split blur pass: LP / 8 lanes per vertex row, lane q owning labels
// 8q .. 8q+7, so that a warp instruction reads whole rows (own and both
// neighbours) instead of one 16-byte piece of 32 rows; a warp holds
// 32 / (LP / 8) rows (lanes beyond that are idle).  Same arithmetic as k_fw_blur.
template <int LP, typename T>
__global__ void __launch_bounds__(256) k_fw_blur3(BlurSet B, int p) {
    constexpr int R = LP / 8;                  // lanes per row
    constexpr int RW = 32 / R;                 // rows per warp
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int r = lane / R, q = lane - R * (lane / R);
    if (r >= RW) return;
    const int64_t g = warp * RW + r;
    if (g >= B.start[B.nk]) return;
    int mm = 0;
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k < B.nk && g >= B.start[k]) mm = k;
    BlurLat lt = B.l[0];
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k == mm) lt = B.l[k];
    if (p >= lt.d1) return;
    const int64_t v = g - B.start[mm];
    const int D = lt.d1 - 1;
    T *out = ((D - p) % 2 == 0) ? (T *)lt.dst : (T *)lt.tmp;
    const int2 nb = reinterpret_cast<const int2 *>(lt.nbr)[v * lt.d1 + p];
    float c[8], a[8], b[8];
    if (p == 0) {
        const float inv = __ldg(lt.qs + 1);
        row_load_q(lt.src0, v, LP, q, inv, c);
        if (nb.x >= 0) row_load_q(lt.src0, nb.x, LP, q, inv, a);
        if (nb.y >= 0) row_load_q(lt.src0, nb.y, LP, q, inv, b);
    } else {
        const T *in = ((D - p + 1) % 2 == 0) ? (const T *)lt.dst : (const T *)lt.tmp;
        row_load<T>(in, v, LP, q, c);
        if (nb.x >= 0) row_load<T>(in, nb.x, LP, q, a);
        if (nb.y >= 0) row_load<T>(in, nb.y, LP, q, b);
    }
    float o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        o[j] = 0.5f * c[j] + (nb.x >= 0 ? 0.25f * a[j] : 0.f) + (nb.y >= 0 ? 0.25f * b[j] : 0.f);
    row_store(out, v, LP, q, o);
}

// Lattice dot products for the line search:
//   0: w s0 sum_v sum_ij mu_ij Ylat[v][i] BS[v][j]   (= <y, K~-part of Psi s>)
//   1: w s0 sum_v sum_ij mu_ij Slat[v][i] BS[v][j]   (= <s, K~-part of Psi s>)
// with Slat = Sq 2^-k the value of the fixed-point splat of s^t, summed per
// warp in FP32.  Before its dot products the kernel brings Ylat up to date:
// Ylat = S y^t = Ylat + alpha_{t-1} (S s^{t-1} - Ylat), S s^{t-1} from Sp,
// which it then clears for the pixel pass's splat of s^{t+1} (alpha_{t-1} = 0
// at the first iteration).  One launch covers every lattice: block b belongs
// to lattice m while start[m] <= b < start[m+1].
struct DotArgs {
    const Chunk *chunks[DCRF_MAX_KERNELS];   // vertex chunks of each lattice
    int start[DCRF_MAX_KERNELS + 1];         // prefix of the chunk counts
    int64_t voff[DCRF_MAX_KERNELS];          // first per-warp row of each lattice
    const double *alpha;                     // [batch] alpha_{t-1}
    const float *mu;
    int L;
    float *vpart;                            // [vertex-chunk warps of all lattices][2] per-warp sums
};

template <int LP, typename T, bool POTTS>
__global__ void __launch_bounds__(kVertBlock) k_fw_latdot(DotArgs A, FwLats F) {
    int mm = 0;
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k < F.nk && (int)blockIdx.x >= A.start[k]) mm = k;
    // the fields of lattice mm (selected one by one: no struct copy in local memory)
    struct {
        float *Ylat;
        uint32_t *Sq, *Sp;
        const void *BS;
        const float *qs;
        const int32_t *vimg;
        float ws0;
    } lt = {F.l[0].Ylat, F.l[0].Sq, F.l[0].Sp, F.l[0].BS, F.l[0].qs, F.l[0].vimg, F.l[0].ws0};
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k == mm) {
            lt.Ylat = F.l[k].Ylat; lt.Sq = F.l[k].Sq; lt.Sp = F.l[k].Sp; lt.BS = F.l[k].BS;
            lt.qs = F.l[k].qs; lt.vimg = F.l[k].vimg; lt.ws0 = F.l[k].ws0;
        }
    int start = A.start[0];
    const Chunk *chunks = A.chunks[0];
    int64_t voff = A.voff[0];
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k == mm) { start = A.start[k]; chunks = A.chunks[k]; voff = A.voff[k]; }
    const int blk = (int)blockIdx.x - start;
    const Chunk ch = chunks[blk];
    float part[2] = {0.f, 0.f};
    if ((int)threadIdx.x < ch.count) {
        const int64_t v = ch.begin + threadIdx.x;
        const float inv = __ldg(lt.qs + 1);
        const float al = (float)A.alpha[lt.vimg[v]];
        float yv[LP], sv[LP], bv[LP];
        // every load of the row is issued before the first store (the stores
        // could alias the loads as far as the compiler knows)
        float4 pv[LP / 4];
#pragma unroll
        for (int g = 0; g < LP / 4; ++g) {
            const int64_t idx = v * (LP / 4) + g;
            const float4 a = ld4(lt.Ylat, idx);
            const float4 b = ld4q(lt.Sq, idx, inv);
            const float4 c = ld4((const T *)lt.BS, idx);
            pv[g] = ld4q(lt.Sp, idx, inv);
            yv[4 * g] = a.x; yv[4 * g + 1] = a.y; yv[4 * g + 2] = a.z; yv[4 * g + 3] = a.w;
            sv[4 * g] = b.x; sv[4 * g + 1] = b.y; sv[4 * g + 2] = b.z; sv[4 * g + 3] = b.w;
            bv[4 * g] = c.x; bv[4 * g + 1] = c.y; bv[4 * g + 2] = c.z; bv[4 * g + 3] = c.w;
        }
#pragma unroll
        for (int g = 0; g < LP / 4; ++g) {
            const int64_t idx = v * (LP / 4) + g;
            float4 a = make_float4(yv[4 * g], yv[4 * g + 1], yv[4 * g + 2], yv[4 * g + 3]);
            a.x += al * (pv[g].x - a.x); a.y += al * (pv[g].y - a.y);
            a.z += al * (pv[g].z - a.z); a.w += al * (pv[g].w - a.w);
            yv[4 * g] = a.x; yv[4 * g + 1] = a.y; yv[4 * g + 2] = a.z; yv[4 * g + 3] = a.w;
            st4(lt.Ylat, idx, a);
            reinterpret_cast<uint4 *>(lt.Sp)[idx] = make_uint4(0u, 0u, 0u, 0u);
        }
        float py = 0.f, ps = 0.f;
        if (POTTS) {
            float ty = 0.f, ts = 0.f, tb = 0.f, dy = 0.f, dsv = 0.f;
#pragma unroll
            for (int i = 0; i < LP; ++i) {
                ty += yv[i]; ts += sv[i]; tb += bv[i];
                dy += yv[i] * bv[i]; dsv += sv[i] * bv[i];
            }
            py = ty * tb - dy;
            ps = ts * tb - dsv;
        } else {
            for (int i = 0; i < A.L; ++i) {
                float mb = 0.f;
#pragma unroll
                for (int j = 0; j < LP; ++j)
                    if (j < A.L) mb += A.mu[i * A.L + j] * bv[j];
                py += yv[i] * mb;
                ps += sv[i] * mb;
            }
        }
        part[0] = lt.ws0 * py;
        part[1] = lt.ws0 * ps;
    }
    warp_sums<2>(part, A.vpart + 2 * (voff + (int64_t)blk * (kVertBlock / 32)));
}

// Per-image FP64 sums of per-chunk FP32 partials: chunks [range[b], range[b+1])
// of rows of width W, summed into out[0 .. W) by the calling block.
struct PartSums {
    const float *cpart;                    // [pixel-chunk warps][NS]
    const int *crange;                     // [batch + 1] rows of cpart per image
    const float *vpart;                    // [vertex-chunk warps of all lattices][2]
    const int *vrange;                     // [nk][batch + 1] rows of vpart per image
    int nk;
    int batch;
};

// Per-image sums of per-warp FP32 partials, compensated FP32 throughout (each
// thread's strided rows, warps, then across warps); each sum becomes FP64
// once, as hi + lo.  rows_into adds rows [r0, r1) of width W into columns
// OFF .. OFF+W of a thread's (hi, lo); block_sums reduces T columns over the
// block, the result valid in thread 0.
template <int W, int OFF, int T>
__device__ __forceinline__ void rows_into(const float *part, int r0, int r1, float (&hi)[T], float (&lo)[T]) {
#pragma unroll 4
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x)
#pragma unroll
        for (int q = 0; q < W; ++q) add_comp(hi[OFF + q], lo[OFF + q], part[(int64_t)r * W + q], 0.f);
}

template <int T>
__device__ __forceinline__ void block_sums(float (&hi)[T], float (&lo)[T], double (&out)[T]) {
    __shared__ float rh[32][T], rl[32][T];
    __shared__ double col[T];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < T; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_down_sync(0xffffffffu, hi[q], o);
            const float l2 = __shfl_down_sync(0xffffffffu, lo[q], o);
            add_comp(hi[q], lo[q], h2, l2);
        }
        if (lane == 0) {
            rh[warp][q] = hi[q];
            rl[warp][q] = lo[q];
        }
    }
    __syncthreads();
    if (threadIdx.x < T) {
        float h = 0.f, l = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) add_comp(h, l, rh[w][threadIdx.x], rl[w][threadIdx.x]);
        col[threadIdx.x] = (double)h + (double)l;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < T; ++q) out[q] = col[q];
}

template <int W>
__device__ __forceinline__ void image_sums(const float *part, int r0, int r1, double (&out)[W]) {
    float hi[W], lo[W];
#pragma unroll
    for (int q = 0; q < W; ++q) hi[q] = lo[q] = 0.f;
    rows_into<W, 0, W>(part, r0, r1, hi, lo);
    block_sums<W>(hi, lo, out);
}

__device__ __forceinline__ void pixel_sums(const PartSums &P, int b, double (&sg)[NS]) {
    image_sums<NS>(P.cpart, P.crange[b], P.crange[b + 1], sg);
}

// Step size and record of one iteration.  kAlphaSplit blocks per image each
// reduce a share of the image's partial rows (compensated FP32, then FP64 as
// hi + lo); the last of them to finish adds the shares in FP64 in block order
// (so the result does not depend on which block finishes last) and writes
// alpha and the record; the last image to finish advances the iteration
// counter.  One block per image left each block with several dependent
// rounds of loads: the kernel took ~15 us at any batch size.
constexpr int kAlphaSplit = 4;

__global__ void __launch_bounds__(1024) k_fw_alpha(PartSums P, double *alpha, dcrf_fw_record *rec, int *counter,
                                                   int *ticket, int *img_ticket, double *share, int *status) {
    const int b = blockIdx.x / kAlphaSplit, j = blockIdx.x - b * kAlphaSplit;
    const int t = *counter;
    // one pass: the pixel sums in columns 0 .. NS-1, the lattice dot products
    // of every lattice in columns NS, NS+1 (they only enter as their total)
    constexpr int T = NS + 2;
    float hi[T], lo[T];
#pragma unroll
    for (int q = 0; q < T; ++q) hi[q] = lo[q] = 0.f;
    // share j of rows [r0, r1)
    auto lo_of = [j](int r0, int r1) { return r0 + (int)((int64_t)(r1 - r0) * j / kAlphaSplit); };
    auto hi_of = [j](int r0, int r1) { return r0 + (int)((int64_t)(r1 - r0) * (j + 1) / kAlphaSplit); };
    {
        const int r0 = P.crange[b], r1 = P.crange[b + 1];
        rows_into<NS, 0, T>(P.cpart, lo_of(r0, r1), hi_of(r0, r1), hi, lo);
    }
#pragma unroll
    for (int m = 0; m < DCRF_MAX_KERNELS; ++m) {
        if (m >= P.nk) break;
        const int *vr = P.vrange + m * (P.batch + 1);
        rows_into<2, NS, T>(P.vpart, lo_of(vr[b], vr[b + 1]), hi_of(vr[b], vr[b + 1]), hi, lo);
    }
    double sg[T];
    block_sums<T>(hi, lo, sg);
    if (threadIdx.x != 0) return;
    double *mine = share + (int64_t)blockIdx.x * T;
#pragma unroll
    for (int q = 0; q < T; ++q) mine[q] = sg[q];
    __threadfence();
    if (atomicAdd(img_ticket + b, 1) != kAlphaSplit - 1) return;
    img_ticket[b] = 0;
    __threadfence();
#pragma unroll
    for (int q = 0; q < T; ++q) sg[q] = 0.0;
    for (int k = 0; k < kAlphaSplit; ++k) {
        const double *sh = share + ((int64_t)b * kAlphaSplit + k) * T;
#pragma unroll
        for (int q = 0; q < T; ++q) sg[q] += __ldcg(sh + q);
    }
    const double yPs = sg[4] + sg[NS], sPs = sg[5] + sg[NS + 1];
    const double A = sPs - sg[3] - yPs + sg[1];
    const double B = sg[2] - sg[0] + yPs - 2.0 * sg[1] + sg[3];
    double al;
    if (!isfinite(A) || !isfinite(B)) {
        dcrf_flag(status, DCRF_E_NONFINITE);
        al = 0.0;
    } else if (A > 0.0) {
        al = fmin(1.0, fmax(0.0, -B / (2.0 * A)));
    } else {
        al = (A + B < 0.0) ? 1.0 : 0.0;
    }
    alpha[b] = al;
    if (rec) {
        dcrf_fw_record r;
        r.energy = sg[0] + sg[1];
        r.gap = sg[0] + 2.0 * sg[1] - sg[2] - 2.0 * sg[3];
        r.alpha = al;
        r.A = A;
        r.B = B;
        rec[(int64_t)t * P.batch + b] = r;
    }
    __threadfence();
    if (atomicAdd(ticket, 1) == P.batch - 1) {
        *ticket = 0;
        *counter = t + 1;
    }
}

// BY += alpha (BS - BY) and its half copy, every lattice in one launch
// (element group idx of lattice m while start[m] <= idx < start[m+1]).
struct UpdArgs {
    int64_t start[DCRF_MAX_KERNELS + 1];   // prefix of m * Lp / 4
    int64_t total;                          // start[nk]
    const double *alpha;
    int G;                                  // Lp / 4
};

template <typename T>
__global__ void k_fw_latupd(FwLats F, UpdArgs U) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= U.total) return;
    int mm = 0;
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k < F.nk && g >= U.start[k]) mm = k;
    float *BY = F.l[0].BY;
    const void *BS = F.l[0].BS;
    __half *BYh = F.l[0].BYh;
    const int32_t *vimg = F.l[0].vimg;
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k == mm) { BY = F.l[k].BY; BS = F.l[k].BS; BYh = F.l[k].BYh; vimg = F.l[k].vimg; }
    int64_t start = U.start[0];
#pragma unroll
    for (int k = 1; k < DCRF_MAX_KERNELS; ++k)
        if (k == mm) start = U.start[k];
    const int64_t idx = g - start;
    const float al = (float)U.alpha[vimg[idx / U.G]];
    float4 by = ld4(BY, idx);
    const float4 bs = ld4((const T *)BS, idx);
    by.x += al * (bs.x - by.x); by.y += al * (bs.y - by.y); by.z += al * (bs.z - by.z); by.w += al * (bs.w - by.w);
    st4(BY, idx, by);
    if (BYh) st4h(BYh, idx, by);
}

// Decision trace: row *counter of trace (when below rows) receives s, the
// conditional gradient the last pixel pass chose (row t = s^t of iteration t).
__global__ void k_fw_trace(const uint8_t *__restrict__ s, uint8_t *__restrict__ trace, const int *counter, int64_t n,
                           int rows) {
    const int t = *counter;
    if (t >= rows) return;
    uint8_t *dst = trace + (int64_t)t * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = s[i];
}

// y^0 must lie on the simplex (rows non-negative, summing to one within
// 1e-5); a row that does not is reported as DCRF_E_INVAL.
__global__ void k_fw_check_y(const float *__restrict__ Y, int64_t n, int L, int *status) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    float sum = 0.f;
    bool ok = true;
    for (int i = 0; i < L; ++i) {
        const float y = Y[a * L + i];
        ok = ok && y >= 0.f;
        sum += y;
    }
    if (!ok || !(fabsf(sum - 1.f) <= 1e-5f)) dcrf_flag(status, DCRF_E_INVAL);
}

// S y^0 in the fixed point of the one-hot splat, so that the solver's state
// does not depend on the order of atomics either: one thread per (point,
// pair of labels) adds round(2^k w y) of both labels of the pair with one
// 64-bit integer reduction (low and high word; a word's sum stays below 2^32,
// since 0 <= y <= 1 bounds it by 2^k (S 1)_v + the roundings, so no carry
// crosses into the other label).
// D1C > 0: d+1 fixed at compile time, every corner's vertex id and weight
// loaded before the first reduction (the loop over runtime d+1 waited on each
// corner's loads in turn).
template <int D1C>
__global__ void k_fw_splat_y0(const float *__restrict__ Y, int64_t n, int L, int Lp, int D1,
                              const int32_t *__restrict__ pvid, const float *__restrict__ pbary, const float *qs,
                              uint32_t *Sq) {
    const int H = Lp >> 1;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * H) return;
    const int64_t a = idx / H;
    const int c0 = 2 * (int)(idx - a * H);
    const float q = __ldg(qs);
    const float y0 = c0 < L ? fmaxf(Y[a * L + c0], 0.f) : 0.f;
    const float y1 = c0 + 1 < L ? fmaxf(Y[a * L + c0 + 1], 0.f) : 0.f;
    if constexpr (D1C > 0) {
        int v[D1C];
        float w[D1C];
#pragma unroll
        for (int k = 0; k < D1C; ++k) {
            v[k] = pvid[a * D1C + k];
            w[k] = pbary[a * D1C + k];
        }
#pragma unroll
        for (int k = 0; k < D1C; ++k) {
            if (v[k] < 0) continue;
            const float wq = q * w[k];
            const unsigned long long lo = __float2uint_rn(wq * y0), hi = __float2uint_rn(wq * y1);
            if (lo | hi)
                atomicAdd(reinterpret_cast<unsigned long long *>(Sq + (int64_t)v[k] * Lp + c0), lo | (hi << 32));
        }
    } else {
        for (int k = 0; k < D1; ++k) {
            const int v = pvid[a * D1 + k];
            if (v < 0) continue;
            const float w = q * pbary[a * D1 + k];
            const unsigned long long lo = __float2uint_rn(w * y0), hi = __float2uint_rn(w * y1);
            if (lo | hi)
                atomicAdd(reinterpret_cast<unsigned long long *>(Sq + (int64_t)v * Lp + c0), lo | (hi << 32));
        }
    }
}

// V = Sq 2^-k as float32.
__global__ void k_fw_dequant(const uint32_t *__restrict__ Sq, int64_t count4, const float *qs, float *V) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count4) st4(V, i, ld4q(Sq, i, __ldg(qs + 1)));
}

__global__ void k_fw_to_half(const float *__restrict__ src, __half *__restrict__ dst, int64_t count4) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count4) st4h(dst, i, ld4(src, i));
}

// c_a = max(0, sum_m w_m (K~_m 1)_a - sum_w);  lin = phi - d  (or phi - 2 d o y)
__global__ void k_fw_c(int64_t n, FwLats F, const float *const *ones, const float *w, int nk, float sumw,
                       float *c) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    float s = 0.f;
    for (int m = 0; m < nk; ++m) s += w[m] * ones[m][a];
    s -= sumw;
    c[a] = s > 0.f ? s : 0.f;
}

// lin = phi - scale musum o c y (y = 1 when Y is null), eight consecutive
// elements of the flat [n][L] arrays per thread: two 16-byte loads of phi
// (and of Y) when the arrays are 16-byte aligned, else eight scalar ones
// (one thread per element kept too few bytes in flight to reach HBM speed).
__device__ __forceinline__ float fw_lin_one(float p, float yv, float scale, const float *musum, const float *c,
                                            int64_t a, int l, int *status) {
    if (!isfinite(p)) dcrf_flag(status, DCRF_E_NONFINITE);
    return p - scale * musum[l] * c[a] * yv;
}

__global__ void k_fw_lin(int64_t n, int L, const float *phi, const float *c, const float *musum,
                         const float *Y, float scale, float *lin, int *status, bool vec) {
    const int64_t count = n * L;
    const int64_t i0 = 8 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    if (i0 >= count) return;
    int64_t a = dcrf_div(i0, L, count);
    int l = (int)(i0 - a * L);
    if (vec && i0 + 8 <= count) {
        float p[8], yv[8], o[8];
        const float4 p0 = reinterpret_cast<const float4 *>(phi + i0)[0], p1 = reinterpret_cast<const float4 *>(phi + i0)[1];
        p[0] = p0.x; p[1] = p0.y; p[2] = p0.z; p[3] = p0.w; p[4] = p1.x; p[5] = p1.y; p[6] = p1.z; p[7] = p1.w;
        if (Y) {
            const float4 y0 = reinterpret_cast<const float4 *>(Y + i0)[0], y1 = reinterpret_cast<const float4 *>(Y + i0)[1];
            yv[0] = y0.x; yv[1] = y0.y; yv[2] = y0.z; yv[3] = y0.w; yv[4] = y1.x; yv[5] = y1.y; yv[6] = y1.z; yv[7] = y1.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) yv[j] = 1.f;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            o[j] = fw_lin_one(p[j], yv[j], scale, musum, c, a, l, status);
            if (++l == L) { l = 0; ++a; }
        }
        reinterpret_cast<float4 *>(lin + i0)[0] = make_float4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<float4 *>(lin + i0)[1] = make_float4(o[4], o[5], o[6], o[7]);
        return;
    }
    const int64_t i1 = i0 + 8 < count ? i0 + 8 : count;
    for (int64_t i = i0; i < i1; ++i) {
        lin[i] = fw_lin_one(phi[i], Y ? Y[i] : 1.f, scale, musum, c, a, l, status);
        if (++l == L) { l = 0; ++a; }
    }
}

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

__global__ void __launch_bounds__(1024) k_fw_qp_energy(PartSums P, double *out) {
    double sg[NS];
    pixel_sums(P, blockIdx.x, sg);
    if (threadIdx.x == 0) out[blockIdx.x] = sg[7] + sg[1] - sg[6];   // phi^T y + y^T (Psi + D) y - y^T D y
}

inline unsigned nblocks(int64_t work, int threads) { return (unsigned)((work + threads - 1) / threads); }

// ---------------------------------------------------------------------------

struct Solver {
    cudaStream_t s;
    Scratch sc;
    int L = 0, Lp = 0, Ls = 0, batch = 0, storage = 0, nk = 0;
    int64_t n = 0;
    bool potts = true;
    float sumw = 0.f;
    const dcrf_lattice *lats = nullptr;
    FwLats F{};
    Chunk *chunks_pb[3] = {nullptr, nullptr, nullptr};   // 256-, 128- and 80-pixel chunk lists
    int n_chunks_pb[3] = {0, 0, 0};
    int variant = -1;                          // chosen pixel-kernel variant
    int blur_variant = -1;                     // chosen blur kernel of every pass, 2 bits per pass
                                               // (0: row per thread, 1: label-split, 2: persistent)
    std::vector<Chunk *> vchunks;
    std::vector<int> n_vchunks;
    float *mu = nullptr, *musum = nullptr, *c = nullptr, *lin = nullptr;
    uint8_t *sidx = nullptr;
    float *cpart = nullptr, *vpart = nullptr;  // per-chunk FP32 partial sums
    int *crange = nullptr;                     // [2][batch + 1] pixel-chunk range per image
    int *vrange = nullptr;                     // [nk][batch + 1] vertex-chunk rows per image
    std::vector<int64_t> voff;                 // first vpart warp row of each lattice
    double *alpha = nullptr;
    int *counter = nullptr, *ticket = nullptr;
    int *img_ticket = nullptr;                 // [batch] blocks of k_fw_alpha done per image
    double *alpha_share = nullptr;             // [batch][kAlphaSplit][NS + 2] their sums
    dcrf_fw_record *rec = nullptr;
    int *status = nullptr;
    uint8_t *trace = nullptr;                  // [trace_rows][n] decisions s^t, or null
    int trace_rows = 0;
    uint32_t *sbuf[DCRF_MAX_KERNELS][2] = {};   // the two one-hot splat buffers of each lattice
    int par = 0;                               // sbuf[m][par] holds S s^t at the start of an iteration

    explicit Solver(cudaStream_t st) : s(st), sc(st) {}

    dcrf_status setup(const float *unaries, const dcrf_lattice *lattices, const float *weights, int n_k,
                      const float *compat, int L_, int store, float *Y, int max_records) {
        DCRF_CHECK_STATUS(dcrf_check_lattices(lattices, n_k));
        if (!unaries || !weights || !Y || L_ < 1 || L_ > DCRF_MAX_L) return DCRF_E_INVAL;
        if (store != DCRF_STORAGE_F32 && store != DCRF_STORAGE_F16) return DCRF_E_INVAL;
        if (L_ > 255) return DCRF_E_INVAL;
        lats = lattices;
        nk = n_k;
        L = L_;
        Lp = L <= 8 ? 8 : (L <= 24 ? 24 : 64);
        Ls = L | 1;
        storage = store;
        n = lattices[0]->n;
        batch = lattices[0]->batch;
        status = lattices[0]->status;
        sumw = 0.f;
        for (int m = 0; m < nk; ++m) {
            if (!(weights[m] >= 0.f)) return DCRF_E_INVAL;
            sumw += weights[m];
        }
        // label compatibility
        std::vector<float> mu_h(L * L), ms_h(L);
        potts = compat == nullptr;
        for (int i = 0; i < L; ++i) {
            float acc_ = 0.f;
            for (int j = 0; j < L; ++j) {
                float v = compat ? compat[i * L + j] : (i == j ? 0.f : 1.f);
                if (!std::isfinite(v)) return DCRF_E_INVAL;
                mu_h[i * L + j] = v;
                acc_ += std::fabs(v);
            }
            ms_h[i] = acc_;
        }
        const size_t esz = storage == DCRF_STORAGE_F16 ? 2 : 4;
        DCRF_CHECK_STATUS(sc.get(&mu, (size_t)L * L));
        DCRF_CHECK_STATUS(sc.get(&musum, (size_t)L));
        DCRF_TRY(cudaMemcpyAsync(mu, mu_h.data(), L * L * sizeof(float), cudaMemcpyHostToDevice, s));
        DCRF_TRY(cudaMemcpyAsync(musum, ms_h.data(), L * sizeof(float), cudaMemcpyHostToDevice, s));
        // lattice workspaces
        F.nk = nk;
        std::vector<int> vrange_h;
        for (int m = 0; m < nk; ++m) {
            FwLat &l = F.l[m];
            const dcrf_lattice lat = lattices[m];
            l.pvid = lat->pvid;
            l.pbary = lat->pbary;
            l.vimg = lat->vimg;
            l.m = lat->m;
            l.d1 = lat->d + 1;
            l.ws0 = (float)(weights[m] * lat->s0);
            const size_t cnt = (size_t)(lat->m > 0 ? lat->m : 1) * Lp;
            DCRF_CHECK_STATUS(sc.get(&l.Ylat, cnt));
            DCRF_CHECK_STATUS(sc.get(&l.BY, cnt));
            DCRF_CHECK_STATUS(sc.get(&sbuf[m][0], cnt));
            DCRF_CHECK_STATUS(sc.get(&sbuf[m][1], cnt));
            DCRF_TRY(cudaMemsetAsync(sbuf[m][1], 0, cnt * sizeof(uint32_t), s));
            l.Sq = l.St = sbuf[m][0];
            l.Sp = sbuf[m][1];
            l.BYh = nullptr;
            if (storage == DCRF_STORAGE_F16) DCRF_CHECK_STATUS(sc.get(&l.BYh, cnt));
            char *bs, *tmp;
            DCRF_CHECK_STATUS(sc.get(&bs, cnt * esz));
            DCRF_CHECK_STATUS(sc.get(&tmp, cnt * esz));
            l.BS = bs;
            l.tmp = tmp;
            DCRF_TRY(cudaMemsetAsync(l.Ylat, 0, cnt * sizeof(float), s));
            DCRF_TRY(cudaMemsetAsync(bs, 0, cnt * esz, s));
            auto ch = make_chunks(lat->vert_off, kVertBlock);
            Chunk *chd = nullptr;
            DCRF_CHECK_STATUS(sc.get(&chd, ch.size() > 0 ? ch.size() : 1));
            if (!ch.empty())
                DCRF_TRY(cudaMemcpyAsync(chd, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice, s));
            vchunks.push_back(chd);
            n_vchunks.push_back((int)ch.size());
            constexpr int vw = kVertBlock / 32;   // warp rows per vertex chunk
            voff.push_back(m == 0 ? 0 : voff[m - 1] + (int64_t)vw * n_vchunks[m - 1]);
            for (int b = 0; b <= batch; ++b) vrange_h.push_back((int)voff[m]);
            for (const Chunk &c : ch) vrange_h[(size_t)m * (batch + 1) + c.image + 1] += vw;
            for (int b = 0; b < batch; ++b)
                vrange_h[(size_t)m * (batch + 1) + b + 1] += vrange_h[(size_t)m * (batch + 1) + b] - (int)voff[m];
        }
        std::vector<int> crange_h(3 * (batch + 1), 0);
        for (int q = 0; q < 3; ++q) {
            auto pc = make_chunks(lattices[0]->point_off, q == 0 ? 256 : (q == 1 ? 128 : kL3Pixels));
            n_chunks_pb[q] = (int)pc.size();
            DCRF_CHECK_STATUS(sc.get(&chunks_pb[q], pc.size() > 0 ? pc.size() : 1));
            if (!pc.empty())
                DCRF_TRY(cudaMemcpyAsync(chunks_pb[q], pc.data(), pc.size() * sizeof(Chunk), cudaMemcpyHostToDevice, s));
            for (const Chunk &c : pc) crange_h[q * (batch + 1) + c.image + 1] += chunk_warps(q);
            for (int b = 0; b < batch; ++b) crange_h[q * (batch + 1) + b + 1] += crange_h[q * (batch + 1) + b];
        }
        const int64_t nv = nk > 0 ? voff[nk - 1] + (int64_t)(kVertBlock / 32) * n_vchunks[nk - 1] : 0;
        int64_t nrows = 1;
        for (int q = 0; q < 3; ++q) nrows = std::max<int64_t>(nrows, (int64_t)chunk_warps(q) * n_chunks_pb[q]);
        DCRF_CHECK_STATUS(sc.get(&cpart, (size_t)nrows * NS));
        DCRF_CHECK_STATUS(sc.get(&vpart, (size_t)std::max<int64_t>(1, nv) * 2));
        DCRF_CHECK_STATUS(sc.get(&crange, crange_h.size()));
        DCRF_CHECK_STATUS(sc.get(&vrange, std::max<size_t>(1, vrange_h.size())));
        DCRF_TRY(cudaMemcpyAsync(crange, crange_h.data(), crange_h.size() * sizeof(int), cudaMemcpyHostToDevice, s));
        if (!vrange_h.empty())
            DCRF_TRY(cudaMemcpyAsync(vrange, vrange_h.data(), vrange_h.size() * sizeof(int), cudaMemcpyHostToDevice,
                                     s));

        DCRF_CHECK_STATUS(sc.get(&c, (size_t)(n > 0 ? n : 1)));
        DCRF_CHECK_STATUS(sc.get(&lin, (size_t)(n > 0 ? n : 1) * L));
        DCRF_CHECK_STATUS(sc.get(&sidx, (size_t)(n > 0 ? n : 1)));
        DCRF_CHECK_STATUS(sc.get(&alpha, (size_t)batch));
        DCRF_TRY(cudaMemsetAsync(alpha, 0, batch * sizeof(double), s));   // no fold is pending at the start
        DCRF_CHECK_STATUS(sc.get(&counter, 2));
        ticket = counter + 1;
        DCRF_CHECK_STATUS(sc.get(&rec, (size_t)batch * (max_records > 0 ? max_records : 1)));
        DCRF_TRY(cudaMemsetAsync(counter, 0, 2 * sizeof(int), s));
        DCRF_CHECK_STATUS(sc.get(&img_ticket, (size_t)batch));
        DCRF_CHECK_STATUS(sc.get(&alpha_share, (size_t)batch * kAlphaSplit * (NS + 2)));
        DCRF_TRY(cudaMemsetAsync(img_ticket, 0, batch * sizeof(int), s));
        // c_a and lin = phi - d
        const float *ones_h[DCRF_MAX_KERNELS];
        for (int m = 0; m < nk; ++m) ones_h[m] = lattices[m]->ones;
        const float **ones_d;
        float *w_d;
        DCRF_CHECK_STATUS(sc.get(&ones_d, nk));
        DCRF_CHECK_STATUS(sc.get(&w_d, nk));
        DCRF_TRY(cudaMemcpyAsync(ones_d, ones_h, nk * sizeof(float *), cudaMemcpyHostToDevice, s));
        DCRF_TRY(cudaMemcpyAsync(w_d, weights, nk * sizeof(float), cudaMemcpyHostToDevice, s));
        if (n > 0) {
            k_fw_c<<<nblocks(n, 256), 256, 0, s>>>(n, F, ones_d, w_d, nk, sumw, c);
            DCRF_LAUNCHED();
            k_fw_lin<<<nblocks((n * L + 7) / 8, 256), 256, 0, s>>>(n, L, unaries, c, musum, nullptr, 1.f, lin, status,
                                                                   aligned16(unaries) && aligned16(lin));
            DCRF_LAUNCHED();
        }
        // fixed-point scales of the one-hot splats: an entry of S s is at most
        // (S 1)_v <= s1max (a bound from the lattice build), so with
        // 2^k (1.001 s1max + 1) <= 2^31 the integer sums cannot overflow
        float *qs_all;
        DCRF_CHECK_STATUS(sc.get(&qs_all, (size_t)2 * nk));
        std::vector<float> qs_h(2 * nk);
        for (int m = 0; m < nk; ++m) {
            const double b = 1.001 * lattices[m]->s1max + 1.0;
            int k = 30;
            while (k > 0 && std::ldexp(b, k) > 2147483648.0) --k;
            qs_h[2 * m] = std::ldexp(1.f, k);
            qs_h[2 * m + 1] = std::ldexp(1.f, -k);
            F.l[m].qs = qs_all + 2 * m;
        }
        DCRF_TRY(cudaMemcpyAsync(qs_all, qs_h.data(), 2 * nk * sizeof(float), cudaMemcpyHostToDevice, s));
        // Ylat = S y0 (fixed point, then float32), BY = B S y0
        if (n > 0) {
            k_fw_check_y<<<nblocks(n, 256), 256, 0, s>>>(Y, n, L, status);
            DCRF_LAUNCHED();
        }
        for (int m = 0; m < nk; ++m) {
            FwLat &l = F.l[m];
            const size_t cnt = (size_t)(l.m > 0 ? l.m : 1) * Lp;
            DCRF_TRY(cudaMemsetAsync(l.Sq, 0, cnt * sizeof(uint32_t), s));
            if (n > 0 && l.m > 0) {
                ProfScope ps(P_SPLAT_DENSE, s);
                const unsigned gb = nblocks(n * (Lp / 2), 256);
                if (l.d1 == 6)
                    k_fw_splat_y0<6><<<gb, 256, 0, s>>>(Y, n, L, Lp, l.d1, l.pvid, l.pbary, l.qs, l.Sq);
                else if (l.d1 == 3)
                    k_fw_splat_y0<3><<<gb, 256, 0, s>>>(Y, n, L, Lp, l.d1, l.pvid, l.pbary, l.qs, l.Sq);
                else
                    k_fw_splat_y0<0><<<gb, 256, 0, s>>>(Y, n, L, Lp, l.d1, l.pvid, l.pbary, l.qs, l.Sq);
                DCRF_LAUNCHED();
                k_fw_dequant<<<nblocks(l.m * Lp / 4, 256), 256, 0, s>>>(l.Sq, l.m * Lp / 4, l.qs, l.Ylat);
                DCRF_LAUNCHED();
            }
            // the splat buffer serves as float32 blur scratch, then is cleared
            DCRF_CHECK_STATUS(dcrf_blur(lattices[m], l.Ylat, l.BY, reinterpret_cast<float *>(l.Sq), Lp,
                                        DCRF_STORAGE_F32, false, s));
            DCRF_TRY(cudaMemsetAsync(l.Sq, 0, cnt * sizeof(uint32_t), s));
            if (l.BYh && l.m > 0) {
                k_fw_to_half<<<nblocks(l.m * Lp / 4, 256), 256, 0, s>>>(l.BY, l.BYh, l.m * Lp / 4);
                DCRF_LAUNCHED();
            }
        }
        return DCRF_OK;
    }

    // Partial-sum layout of the chosen pixel variant (after the first pixel pass).
    PartSums parts() const {
        PartSums P;
        const int q = chunk_list(kPixPB[variant < 0 ? 0 : variant]);
        P.cpart = cpart;
        P.crange = crange + q * (batch + 1);
        P.vpart = vpart;
        P.vrange = vrange;
        P.nk = nk;
        P.batch = batch;
        return P;
    }

    template <int LPc, typename T, bool POT, int PB, int MB, int MODE>
    dcrf_status pixel_v(float *Y, const float *phi, bool start, const double *alpha_override = nullptr) {
        PixArgs A;
        const int q = chunk_list(PB);
        A.chunks = chunks_pb[q];
        A.alpha = start ? nullptr : (alpha_override ? alpha_override : alpha);
        A.Y = Y;
        A.lin = lin;
        A.phi = phi;
        A.s = sidx;
        A.c = c;
        A.mu = mu;
        A.musum = musum;
        A.sumw = sumw;
        A.L = L;
        A.Ls = Ls;
        A.y16 = (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
        A.cpart = cpart;
        A.status = status;
        const size_t shm = 2 * (size_t)PB * Ls * sizeof(float);
        void (*kern)(PixArgs, FwLats);
        int threads = PB;
        if constexpr ((MODE & kL3) != 0) {
            static_assert(LPc == 24 && POT && PB == kL3Pixels, "label-split layout: 24 padded labels, Potts");
            kern = k_fw_pixel3<T>;
            threads = 32 * kL3Warps;
        } else {
            kern = k_fw_pixel<LPc, T, POT, PB, MB, MODE>;
        }
        // the row stride (and so the tile) grows with L: raise the limit when needed
        static int attr_shm = 0;
        if ((int)shm > attr_shm) {
            DCRF_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
            attr_shm = (int)shm;
        }
        if (n_chunks_pb[q] > 0) {
            ProfScope ps(P_FW_PIXEL, s);
            kern<<<n_chunks_pb[q], threads, shm, s>>>(A, F);
            DCRF_LAUNCHED();
        }
        return DCRF_OK;
    }

    // Only the common case (up to 24 labels, Potts) is compiled in every
    // variant; the others use the first one.
    template <int LPc, typename T, bool POT>
    dcrf_status pixel_var(int v, float *Y, const float *phi, bool start, const double *al = nullptr) {
        if constexpr (LPc == 24 && POT) {
#define DCRF_PIX_CASE(V) \
    case V: return pixel_v<LPc, T, POT, kPixPB[V], kPixMB[V], kPixMode[V]>(Y, phi, start, al)
            switch (v) {
                DCRF_PIX_CASE(1);
                DCRF_PIX_CASE(2);
                DCRF_PIX_CASE(3);
                DCRF_PIX_CASE(4);
                DCRF_PIX_CASE(5);
                DCRF_PIX_CASE(6);
                DCRF_PIX_CASE(7);
                DCRF_PIX_CASE(8);
                DCRF_PIX_CASE(9);
                DCRF_PIX_CASE(10);
                DCRF_PIX_CASE(11);
                DCRF_PIX_CASE(12);
                DCRF_PIX_CASE(13);
                DCRF_PIX_CASE(14);
                DCRF_PIX_CASE(15);
                DCRF_PIX_CASE(16);
                DCRF_PIX_CASE(17);
                DCRF_PIX_CASE(18);
            default: return pixel_v<LPc, T, POT, kPixPB[0], kPixMB[0], kPixMode[0]>(Y, phi, start, al);
            }
#undef DCRF_PIX_CASE
        } else {
            (void)v;
            return pixel_v<LPc, T, POT, kPixPB[0], (LPc <= 24 ? kPixMB[0] : 2), 0>(Y, phi, start, al);
        }
    }

    // Autotuner: times every variant on this problem as a full iteration with
    // a zero step (y' = y exactly, so y is rewritten unchanged; s, the splat
    // and the scalar sums are reset afterwards) and keeps the fastest per
    // (Lp, storage, Potts, size bucket).
    template <int LPc, typename T, bool POT>
    dcrf_status tune(const float *Y) {
        if (const char *force = std::getenv("DCRF_PIXEL_VARIANT")) {   // testing hook
            const int v = std::atoi(force);
            variant = (LPc == 24 && POT && v >= 0 && v < kPixVariants && pixel_variant_fits(v, L)) ? v : 0;
            return DCRF_OK;
        }
        static std::mutex mu_;
        static std::map<std::tuple<int, int, int, bool, int>, int> cache;
        int bucket = 0;
        while ((int64_t)1 << (bucket + 1) <= n) ++bucket;
        const auto key = std::make_tuple(LPc, L, storage, POT, bucket);
        {
            std::lock_guard<std::mutex> lk(mu_);
            auto it = cache.find(key);
            if (it != cache.end()) { variant = it->second; return DCRF_OK; }
        }
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        DCRF_TRY(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone || n < 4096 || !(LPc == 24 && POT)) { variant = 0; return DCRF_OK; }
        double *zero = nullptr;
        DCRF_CHECK_STATUS(sc.get(&zero, (size_t)batch));
        DCRF_TRY(cudaMemsetAsync(zero, 0, batch * sizeof(double), s));
        cudaEvent_t e0, e1;
        DCRF_TRY(cudaEventCreate(&e0));
        DCRF_TRY(cudaEventCreate(&e1));
        float best = 1e30f;
        int arg = 0;
        float *Yw = const_cast<float *>(Y);
        for (int v = 0; v < kPixVariants; ++v) {
            if (!pixel_variant_fits(v, L)) continue;
            DCRF_CHECK_STATUS((pixel_var<LPc, T, POT>(v, Yw, nullptr, false, zero)));   // warm-up
            DCRF_TRY(cudaEventRecord(e0, s));
            for (int r = 0; r < 3; ++r) DCRF_CHECK_STATUS((pixel_var<LPc, T, POT>(v, Yw, nullptr, false, zero)));
            DCRF_TRY(cudaEventRecord(e1, s));
            DCRF_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            DCRF_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (std::getenv("DCRF_TUNE_LOG"))
                std::fprintf(stderr, "dcrf tune: Lp=%d storage=%d n=%lld variant %d: %.1f us\n", LPc, storage,
                             (long long)n, v, 1000.f * ms / 3.f);
            if (ms < best) { best = ms; arg = v; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (int m = 0; m < nk; ++m)
            DCRF_TRY(cudaMemsetAsync(F.l[m].St, 0, (size_t)(F.l[m].m > 0 ? F.l[m].m : 1) * Lp * sizeof(uint32_t), s));
        variant = arg;
        std::lock_guard<std::mutex> lk(mu_);
        cache[key] = arg;
        return DCRF_OK;
    }

    template <int LPc, typename T, bool POT>
    dcrf_status pixel_t(float *Y, const float *phi, bool start) {
        if (variant < 0) DCRF_CHECK_STATUS((tune<LPc, T, POT>(Y)));
        return pixel_var<LPc, T, POT>(variant, Y, phi, start);
    }

    template <typename T, bool POT>
    dcrf_status pixel_lp(float *Y, const float *phi, bool start) {
        if (Lp == 8) return pixel_t<8, T, POT>(Y, phi, start);
        if (Lp == 24) return pixel_t<24, T, POT>(Y, phi, start);
        return pixel_t<64, T, POT>(Y, phi, start);
    }

    // Splat buffers of this step: Sq = S s^t, Sp = S s^{t-1} (folded and
    // cleared by the line-search kernel), St = the pixel pass's target.
    void bind(bool start) {
        for (int m = 0; m < nk; ++m) {
            F.l[m].Sq = sbuf[m][par];
            F.l[m].Sp = sbuf[m][par ^ 1];
            F.l[m].St = start ? sbuf[m][par] : sbuf[m][par ^ 1];
        }
    }

    dcrf_status pixel(float *Y, const float *phi, bool start) {
        bind(start);
        dcrf_status st;
        if (storage == DCRF_STORAGE_F16)
            st = potts ? pixel_lp<__half, true>(Y, phi, start) : pixel_lp<__half, false>(Y, phi, start);
        else
            st = potts ? pixel_lp<float, true>(Y, phi, start) : pixel_lp<float, false>(Y, phi, start);
        if (st != DCRF_OK || !trace || n == 0) return st;
        k_fw_trace<<<(unsigned)std::min<int64_t>(nblocks(n, 256), 4096), 256, 0, s>>>(sidx, trace, counter, n,
                                                                                      trace_rows);
        DCRF_LAUNCHED();
        return DCRF_OK;
    }

    // d+1 Jacobi passes of S s (Sq) into BS for every lattice, one launch per pass
    // (tune_only: pick the blur kernel, as run() does before graph capture).
    template <int LPc, typename T>
    dcrf_status blur_t(bool tune_only = false) {
        BlurSet B{};
        B.nk = nk;
        // lattices in order of decreasing d+1, so the ones still blurring at
        // pass p are a prefix of the vertex range
        int order[DCRF_MAX_KERNELS];
        for (int m = 0; m < nk; ++m) order[m] = m;
        std::sort(order, order + nk, [&](int a, int b) { return F.l[a].d1 > F.l[b].d1; });
        B.start[0] = 0;
        for (int k = 0; k < nk; ++k) {
            const int m = order[k];
            B.l[k].nbr = lats[m]->nbr;
            B.l[k].src0 = F.l[m].Sq;
            B.l[k].qs = F.l[m].qs;
            B.l[k].dst = F.l[m].BS;
            B.l[k].tmp = F.l[m].tmp;
            B.l[k].m = F.l[m].m;
            B.l[k].d1 = F.l[m].d1;
            B.start[k + 1] = B.start[k] + F.l[m].m;
        }
        const int dmax = nk > 0 ? B.l[0].d1 : 0;
        if (blur_variant < 0) DCRF_CHECK_STATUS((tune_blur<LPc, T>(B, dmax)));
        if (tune_only) return DCRF_OK;
        return blur_passes<LPc, T>(B, dmax, blur_variant);
    }

    template <int LPc, typename T>
    dcrf_status blur_passes(const BlurSet &B, int dmax, int code) {
        for (int p = 0; p < dmax; ++p) DCRF_CHECK_STATUS((blur_pass<LPc, T>(B, p, (code >> (2 * p)) & 3)));
        return DCRF_OK;
    }

    // Jacobi pass p of every lattice that has it, with blur kernel variant_.
    template <int LPc, typename T>
    dcrf_status blur_pass(const BlurSet &B, int p, int variant_) {
        {
            int active = 0;
            while (active < nk && B.l[active].d1 > p) ++active;
            const int64_t work = B.start[active];
            if (work == 0) return DCRF_OK;
            ProfScope ps(P_FW_BLUR, s);
            if (variant_ == 1) {
                constexpr int RW = 32 / (LPc / 8);
                const int64_t warps = (work + RW - 1) / RW;
                k_fw_blur3<LPc, T><<<nblocks(warps * 32, 256), 256, 0, s>>>(B, p);
            } else if (variant_ == 2) {
                const int64_t full = (work + 255) / 256;
                const int64_t grid = std::min<int64_t>(full, (int64_t)resident_blocks<LPc, T>());
                k_fw_blur2<LPc, T><<<(unsigned)grid, 256, 0, s>>>(B, p, work);
            } else {
                k_fw_blur<LPc, T><<<nblocks(work, 256), 256, 0, s>>>(B, p);
            }
            DCRF_LAUNCHED();
        }
        return DCRF_OK;
    }

    // Blocks of k_fw_blur2 that fit on the device at once (SMs x resident blocks per SM).
    template <int LPc, typename T>
    int resident_blocks() {
        static int cached = 0;
        if (cached > 0) return cached;
        int dev = 0, sms = 1, per_sm = 1;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fw_blur2<LPc, T>, 256, 0) != cudaSuccess)
            return 1024;
        cached = std::max(1, sms * std::max(1, per_sm));
        return cached;
    }

    // Blur tuner: a vertex row per thread (0), label-split rows (1) or the
    // persistent form with the neighbour pair loaded a row ahead (2), timed
    // pass by pass on this problem's lattices (the blur only reads Sq and
    // writes BS and tmp, which every iteration overwrites; the passes that
    // only the higher-dimensional lattice has are smaller and can favour
    // another kernel) and cached per (Lp, storage, size bucket).
    static int blur_code_all(int v) {
        int code = 0;
        for (int p = 0; p < DCRF_MAX_D + 1; ++p) code |= v << (2 * p);
        return code;
    }

    template <int LPc, typename T>
    dcrf_status tune_blur(const BlurSet &B, int dmax) {
        if (const char *force = std::getenv("DCRF_BLUR_VARIANT")) {   // testing hook
            const int f = std::atoi(force);
            blur_variant = blur_code_all((f == 1 || f == 2) ? f : 0);
            return DCRF_OK;
        }
        static std::mutex mu_;
        static std::map<std::tuple<int, int, int>, int> cache;
        const int64_t work = B.start[nk];
        int bucket = 0;
        while ((int64_t)1 << (bucket + 1) <= work) ++bucket;
        const auto key = std::make_tuple(LPc, storage, bucket);
        {
            std::lock_guard<std::mutex> lk(mu_);
            auto it = cache.find(key);
            if (it != cache.end()) { blur_variant = it->second; return DCRF_OK; }
        }
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        DCRF_TRY(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone || work < 4096) { blur_variant = 0; return DCRF_OK; }
        cudaEvent_t e0, e1;
        DCRF_TRY(cudaEventCreate(&e0));
        DCRF_TRY(cudaEventCreate(&e1));
        int arg = 0;
        for (int p = 0; p < dmax; ++p) {
            float best = 1e30f;
            int bv = 0;
            for (int v = 0; v < 3; ++v) {
                DCRF_CHECK_STATUS((blur_pass<LPc, T>(B, p, v)));   // warm-up
                DCRF_TRY(cudaEventRecord(e0, s));
                for (int r = 0; r < 3; ++r) DCRF_CHECK_STATUS((blur_pass<LPc, T>(B, p, v)));
                DCRF_TRY(cudaEventRecord(e1, s));
                DCRF_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                DCRF_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (std::getenv("DCRF_TUNE_LOG"))
                    std::fprintf(stderr, "dcrf tune: blur Lp=%d storage=%d rows=%lld pass %d variant %d: %.1f us\n",
                                 LPc, storage, (long long)work, p, v, 1000.f * ms / 3.f);
                if (ms < best) { best = ms; bv = v; }
            }
            arg |= bv << (2 * p);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        blur_variant = arg;
        std::lock_guard<std::mutex> lk(mu_);
        cache[key] = arg;
        return DCRF_OK;
    }

    dcrf_status blur_all(bool tune_only = false) {
        if (storage == DCRF_STORAGE_F16) {
            if (Lp == 8) return blur_t<8, __half>(tune_only);
            if (Lp == 24) return blur_t<24, __half>(tune_only);
            return blur_t<64, __half>(tune_only);
        }
        if (Lp == 8) return blur_t<8, float>(tune_only);
        if (Lp == 24) return blur_t<24, float>(tune_only);
        return blur_t<64, float>(tune_only);
    }

    template <int LPc, typename T, bool POT>
    dcrf_status latdot_t() {
        DotArgs A{};
        A.start[0] = 0;
        for (int m = 0; m < nk; ++m) {
            A.chunks[m] = vchunks[m];
            A.start[m + 1] = A.start[m] + n_vchunks[m];
            A.voff[m] = voff[m];
        }
        A.alpha = alpha;
        A.mu = mu;
        A.L = L;
        A.vpart = vpart;
        if (A.start[nk] > 0) {
            ProfScope ps(P_FW_LATDOT, s);
            k_fw_latdot<LPc, T, POT><<<A.start[nk], kVertBlock, 0, s>>>(A, F);
            DCRF_LAUNCHED();
        }
        return DCRF_OK;
    }

    template <typename T, bool POT>
    dcrf_status latdot_lp() {
        if (Lp == 8) return latdot_t<8, T, POT>();
        if (Lp == 24) return latdot_t<24, T, POT>();
        return latdot_t<64, T, POT>();
    }

    dcrf_status latdot() {
        if (storage == DCRF_STORAGE_F16)
            return potts ? latdot_lp<__half, true>() : latdot_lp<__half, false>();
        return potts ? latdot_lp<float, true>() : latdot_lp<float, false>();
    }

    // One Frank-Wolfe iteration, state at (y^t, s^t, Sq = S s^t, BY = B S y^t,
    // Ylat + alpha_{t-1} (S s^{t-1} - Ylat) = S y^t with S s^{t-1} in Sp).
    dcrf_status iterate(float *Y, const float *phi) {
        bind(false);
        DCRF_CHECK_STATUS(blur_all());
        DCRF_CHECK_STATUS(latdot());
        {
            ProfScope ps(P_FW_ALPHA, s);
            k_fw_alpha<<<batch * kAlphaSplit, 1024, 0, s>>>(parts(), alpha, rec, counter, ticket, img_ticket,
                                                           alpha_share, status);
        }
        DCRF_LAUNCHED();
        UpdArgs U{};
        U.G = Lp / 4;
        U.alpha = alpha;
        U.start[0] = 0;
        for (int m = 0; m < nk; ++m) U.start[m + 1] = U.start[m] + F.l[m].m * U.G;
        U.total = U.start[nk];
        if (U.start[nk] > 0) {
            ProfScope ps(P_FW_LATUPD, s);
            if (storage == DCRF_STORAGE_F16)
                k_fw_latupd<__half><<<nblocks(U.start[nk], 256), 256, 0, s>>>(F, U);
            else
                k_fw_latupd<float><<<nblocks(U.start[nk], 256), 256, 0, s>>>(F, U);
            DCRF_LAUNCHED();
        }
        DCRF_CHECK_STATUS(pixel(Y, phi, false));
        par ^= 1;   // the splat of s^{t+1} is the next iteration's S s
        return DCRF_OK;
    }

    // Runs `iters` iterations; uses a CUDA graph of two iterations when the
    // stream allows capture.
    dcrf_status run(float *Y, int iters, const float *phi_last) {
        int done = 0;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        DCRF_TRY(cudaStreamIsCapturing(s, &cs));
        const bool graph_ok = s != nullptr && cs == cudaStreamCaptureStatusNone && iters >= 6 && !dcrf_profiling();
        if (iters > 0 && blur_variant < 0) DCRF_CHECK_STATUS(blur_all(true));   // tune outside the capture
        if (graph_ok) {
            cudaGraph_t g = nullptr;
            DCRF_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            dcrf_status st = iterate(Y, nullptr);
            if (st == DCRF_OK) st = iterate(Y, nullptr);
            cudaError_t e = cudaStreamEndCapture(s, &g);
            if (st != DCRF_OK) { if (g) cudaGraphDestroy(g); return st; }
            if (e != cudaSuccess) return DCRF_E_CUDA;
            cudaGraphExec_t ge = nullptr;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return DCRF_E_CUDA;
            const int pairs = (iters - 1) / 2;
            for (int p = 0; p < pairs; ++p) {
                e = cudaGraphLaunch(ge, s);
                if (e != cudaSuccess) { cudaGraphExecDestroy(ge); return DCRF_E_CUDA; }
            }
            cudaGraphExecDestroy(ge);
            done = 2 * pairs;
        }
        for (int t = done; t < iters; ++t) DCRF_CHECK_STATUS(iterate(Y, t == iters - 1 ? phi_last : nullptr));
        return DCRF_OK;
    }
};

}  // namespace

extern "C" dcrf_status dcrf_qp_fw_trace(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                        int n_kernels, const float *compat, int L, int iters, float *Y,
                                        dcrf_fw_record *records, uint8_t *s_trace, int storage,
                                        dcrf_stream stream) {
    if (iters < 0) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Solver S(s);
    DCRF_CHECK_STATUS(S.setup(unaries, lattices, weights, n_kernels, compat, L, storage, Y, iters));
    if (S.n == 0) return DCRF_OK;
    S.trace = s_trace;
    S.trace_rows = iters;
    DCRF_CHECK_STATUS(S.pixel(Y, nullptr, true));
    DCRF_CHECK_STATUS(S.run(Y, iters, nullptr));
    if (records && iters > 0) {
        DCRF_TRY(cudaMemcpyAsync(records, S.rec, (size_t)iters * S.batch * sizeof(dcrf_fw_record),
                                 cudaMemcpyDeviceToHost, s));
        int h = 0;
        DCRF_TRY(cudaMemcpyAsync(&h, S.status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DCRF_TRY(cudaStreamSynchronize(s));
        if (h != 0) return (dcrf_status)h;
    }
    return DCRF_OK;
}

namespace {

// Test of the bounded mbarrier wait that the pixel pass uses for its tile
// copies: one block arms an mbarrier and polls it `polls` times.  With
// never_complete, the barrier expects 16 bytes that no copy delivers (nothing
// is in flight), so the wait runs out and DCRF_E_TIMEOUT is flagged;
// otherwise the phase completes at once.  The barrier is invalidated before
// the block exits.
__global__ void k_wait_selftest(int *status, long long polls, int never_complete) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        if (never_complete) mbar_expect_tx(&bar, 16u);
        else mbar_arrive(&bar);
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, polls);
    if (__syncthreads_and(ok) == 0 && threadIdx.x == 0) dcrf_flag(status, DCRF_E_TIMEOUT);
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(&bar);
}

}  // namespace

extern "C" dcrf_status dcrf_selftest_bounded_wait(dcrf_lattice lat, int64_t polls, int never_complete,
                                                  dcrf_stream stream) {
    if (!lat || polls < 1 || polls > (1ll << 26)) return DCRF_E_INVAL;
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(lat->status, (long long)polls, never_complete ? 1 : 0);
    DCRF_LAUNCHED();
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_qp_fw(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                  int n_kernels, const float *compat, int L, int iters, float *Y,
                                  dcrf_fw_record *records, int storage, dcrf_stream stream) {
    return dcrf_qp_fw_trace(unaries, lattices, weights, n_kernels, compat, L, iters, Y, records, nullptr, storage,
                            stream);
}

extern "C" dcrf_status dcrf_dc_cccp_trace(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                          int n_kernels, const float *compat, int L, int outer, int inner, float *Y,
                                          double *qp_energy, uint8_t *s_trace, int storage, dcrf_stream stream) {
    if (outer < 0 || inner < 0) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Solver S(s);
    DCRF_CHECK_STATUS(S.setup(unaries, lattices, weights, n_kernels, compat, L, storage, Y, outer * inner));
    if (S.n == 0) return DCRF_OK;
    // row o * inner + i: the decision of inner iteration i of outer step o
    // (each outer step's start pass rewrites the row the previous step's last
    // pass wrote, with the new linear term)
    S.trace = s_trace;
    S.trace_rows = outer * inner;
    double *qe;
    DCRF_CHECK_STATUS(S.sc.get(&qe, (size_t)(outer + 1) * S.batch));
    // S_QP at y^0
    DCRF_CHECK_STATUS(S.pixel(Y, unaries, true));
    k_fw_qp_energy<<<S.batch, 1024, 0, s>>>(S.parts(), qe);
    DCRF_LAUNCHED();
    const int G = S.Lp / 4;
    (void)G;
    for (int o = 0; o < outer; ++o) {
        // linearise q at y^t: lin = phi - 2 d o y^t
        k_fw_lin<<<nblocks((S.n * L + 7) / 8, 256), 256, 0, s>>>(S.n, L, unaries, S.c, S.musum, Y, 2.f, S.lin, S.status,
                                                                 aligned16(unaries) && aligned16(Y) && aligned16(S.lin));
        DCRF_LAUNCHED();
        for (int m = 0; m < S.nk; ++m)
            DCRF_TRY(cudaMemsetAsync(S.sbuf[m][S.par], 0,
                                     (size_t)(S.F.l[m].m > 0 ? S.F.l[m].m : 1) * S.Lp * sizeof(uint32_t), s));
        DCRF_CHECK_STATUS(S.pixel(Y, inner == 0 ? unaries : nullptr, true));
        DCRF_CHECK_STATUS(S.run(Y, inner, unaries));
        k_fw_qp_energy<<<S.batch, 1024, 0, s>>>(S.parts(), qe + (int64_t)(o + 1) * S.batch);
        DCRF_LAUNCHED();
    }
    if (qp_energy) {
        DCRF_TRY(cudaMemcpyAsync(qp_energy, qe, (size_t)(outer + 1) * S.batch * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
        int h = 0;
        DCRF_TRY(cudaMemcpyAsync(&h, S.status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DCRF_TRY(cudaStreamSynchronize(s));
        if (h != 0) return (dcrf_status)h;
    }
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_dc_cccp(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                    int n_kernels, const float *compat, int L, int outer, int inner, float *Y,
                                    double *qp_energy, int storage, dcrf_stream stream) {
    return dcrf_dc_cccp_trace(unaries, lattices, weights, n_kernels, compat, L, outer, inner, Y, qp_energy, nullptr,
                              storage, stream);
}

namespace {

// ---------------------------------------------------------------------------
// CCCP for negative semi-definite compatibilities (Section 5.2, Appendix C).
//
// S_QP(y) = [phi^T y - sum_w y^T (mu (x) I) y] + [y^T (mu (x) K~) y]: convex
// plus concave on M.  Each outer step needs one filter of y^t: the gradient
// of the concave part is mu (K~ y + K~^T y), and since K~ = S^T B S and
// K~^T = S^T B^T S (B^T: the blur axes in reverse order), one splat of y feeds
// the forward and the reverse blur and a single slice of their sum.  The
// convex problem then decouples over pixels:
//   min_{y_a in simplex} lin_a^T y_a - sum_w y_a^T mu y_a,
//   lin_a = phi_a + mu (K~ y^t + K~^T y^t)_a.
// Potts: the minimiser is the Euclidean projection of -lin_a / (2 sum_w)
// (Michelot's active-set iteration); other symmetric mu: `inner` per-pixel
// Frank-Wolfe steps with the exact step, from y^t_a.  The same pass sums
// S_QP(y^t) = phi^T y + 1/2 y^T mu F - sum_w y^T mu y, F = K~ y + K~^T y.

struct NegLat {
    const int32_t *pvid;
    const float *pbary;
    const void *V1;    // [m][Lp] B S y   (storage type)
    const void *V2;    // [m][Lp] B^T S y (storage type)
    int d1;
    float ws0;
};

struct NegArgs {
    const Chunk *chunks;   // 256-pixel chunks
    NegLat l[DCRF_MAX_KERNELS];
    int nk;
    float *Y;              // [n][L] in/out
    const float *phi;      // [n][L]
    const float *mu;       // [L][L] (general mu)
    int L;
    int inner;
    bool update;           // false: energy only
    bool mf;               // mean-field update instead of the CCCP step
    float sumw;
    float *epart;          // [chunks][8 warps] per-warp S_QP sums
    int *status;
};

template <int LP, typename TB, bool POTTS>
__global__ void __launch_bounds__(256) k_dcneg_pixel(NegArgs A) {
    const Chunk ch = A.chunks[blockIdx.x];
    const int t = threadIdx.x;
    const bool valid = t < ch.count;
    const int64_t a = ch.begin + (valid ? t : 0);
    const int L = A.L;
    float e = 0.f;
    if (valid) {
        // F = sum_m w_m s0_m S_m^T (B_m + B_m^T) S_m y, eight labels at a time
        float F[LP];
#pragma unroll
        for (int i = 0; i < LP; ++i) F[i] = 0.f;
#pragma unroll
        for (int mm = 0; mm < DCRF_MAX_KERNELS; ++mm) {
            if (mm >= A.nk) break;
            const NegLat &lt = A.l[mm];
            for (int k = 0; k < lt.d1; ++k) {
                const int v = __ldg(lt.pvid + a * lt.d1 + k);
                if (v < 0) continue;
                const float w = __ldg(lt.pbary + a * lt.d1 + k) * lt.ws0;
#pragma unroll
                for (int h = 0; h < LP / 8; ++h) {
                    float o1[8], o2[8];
                    ld8((const TB *)lt.V1, v, LP, h, o1);
                    ld8((const TB *)lt.V2, v, LP, h, o2);
#pragma unroll
                    for (int j = 0; j < 8; ++j) F[8 * h + j] += w * (o1[j] + o2[j]);
                }
            }
        }
        float y[LP], ph[LP], muF[LP], muy[LP];
#pragma unroll
        for (int i = 0; i < LP; ++i) {
            y[i] = i < L ? A.Y[a * L + i] : 0.f;
            ph[i] = i < L ? A.phi[a * L + i] : 0.f;
        }
        if (POTTS) {
            float tF = 0.f, ty = 0.f;
#pragma unroll
            for (int i = 0; i < LP; ++i)
                if (i < L) { tF += F[i]; ty += y[i]; }
#pragma unroll
            for (int i = 0; i < LP; ++i) {
                muF[i] = tF - F[i];
                muy[i] = ty - y[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < LP; ++i) {
                float sf = 0.f, sy = 0.f;
                if (i < L) {
#pragma unroll 8
                    for (int j = 0; j < LP; ++j)
                        if (j < L) {
                            const float m = A.mu[i * L + j];
                            sf += m * F[j];
                            sy += m * y[j];
                        }
                }
                muF[i] = sf;
                muy[i] = sy;
            }
        }
#pragma unroll
        for (int i = 0; i < LP; ++i)
            if (i < L) e += ph[i] * y[i] + 0.5f * y[i] * muF[i] - A.sumw * y[i] * muy[i];
        if (A.update && A.mf) {
            // mean field: Q = softmax(-phi - (Psi + Psi^T) Q),
            // (Psi + Psi^T) Q = mu F - 2 sum_w mu Q   (mu symmetric)
            float z[LP], zmax = -INFINITY;
#pragma unroll
            for (int i = 0; i < LP; ++i) {
                z[i] = -ph[i] - muF[i] + 2.f * A.sumw * muy[i];
                if (i < L) {
                    if (!isfinite(z[i])) dcrf_flag(A.status, DCRF_E_NONFINITE);
                    zmax = fmaxf(zmax, z[i]);
                }
            }
            float den = 0.f;
#pragma unroll
            for (int i = 0; i < LP; ++i) {
                z[i] = i < L ? expf(z[i] - zmax) : 0.f;
                den += z[i];
            }
            const float inv = 1.f / den;
#pragma unroll
            for (int i = 0; i < LP; ++i)
                if (i < L) A.Y[a * L + i] = z[i] * inv;
        } else if (A.update) {
            float lin[LP];
#pragma unroll
            for (int i = 0; i < LP; ++i) lin[i] = ph[i] + muF[i];
            if (POTTS) {
                // projection of v = -lin / (2 sum_w) onto the simplex; the
                // projection is unchanged by a shift of v, and shifting by
                // max v keeps tau small so that v - tau does not cancel
                const float sc = -0.5f / A.sumw;
                float v[LP];
                bool act[LP];
                float vmax = -INFINITY;
#pragma unroll
                for (int i = 0; i < LP; ++i) {
                    v[i] = lin[i] * sc;
                    act[i] = i < L;
                    if (i < L) {
                        if (!isfinite(v[i])) dcrf_flag(A.status, DCRF_E_NONFINITE);
                        vmax = fmaxf(vmax, v[i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < LP; ++i) v[i] -= vmax;
                float tau = 0.f;
                for (int it = 0; it <= L; ++it) {
                    float sm = 0.f;
                    int cnt = 0;
#pragma unroll
                    for (int i = 0; i < LP; ++i)
                        if (act[i]) { sm += v[i]; ++cnt; }
                    tau = (sm - 1.f) / (float)cnt;
                    bool changed = false;
#pragma unroll
                    for (int i = 0; i < LP; ++i)
                        if (act[i] && v[i] <= tau) { act[i] = false; changed = true; }
                    if (!changed) break;
                }
#pragma unroll
                for (int i = 0; i < LP; ++i) y[i] = act[i] ? v[i] - tau : 0.f;
            } else {
                // Frank-Wolfe on lin^T y - sum_w y^T mu y (mu symmetric): gradient
                // lin - 2 sum_w mu y, exact step on the per-pixel quadratic
                for (int it = 0; it < A.inner; ++it) {
                    float g[LP];
                    float best = INFINITY;
                    int sb = 0;
#pragma unroll
                    for (int i = 0; i < LP; ++i) {
                        g[i] = lin[i] - 2.f * A.sumw * muy[i];
                        if (i < L && g[i] < best) { best = g[i]; sb = i; }
                    }
                    if (!(best < INFINITY)) { dcrf_flag(A.status, DCRF_E_NONFINITE); break; }
                    // d = e_sb - y:  d^T mu d = mu_ss - 2 (mu y)_s + y^T mu y,  g^T d = g_s - g^T y
                    float ymy = 0.f, gy = 0.f;
#pragma unroll
                    for (int i = 0; i < LP; ++i)
                        if (i < L) { ymy += y[i] * muy[i]; gy += g[i] * y[i]; }
                    float muys = 0.f, gs = 0.f;
#pragma unroll
                    for (int i = 0; i < LP; ++i)
                        if (i == sb) { muys = muy[i]; gs = g[i]; }
                    const float dmd = A.mu[sb * L + sb] - 2.f * muys + ymy;
                    const float qa = -A.sumw * dmd, qb = gs - gy;
                    float al;
                    if (qa > 0.f) al = fminf(1.f, fmaxf(0.f, -qb / (2.f * qa)));
                    else al = (qa + qb < 0.f) ? 1.f : 0.f;
                    // y += al (e_s - y); mu y += al (mu e_s - mu y)
#pragma unroll
                    for (int i = 0; i < LP; ++i) {
                        if (i < L) {
                            y[i] += al * ((i == sb ? 1.f : 0.f) - y[i]);
                            muy[i] += al * (A.mu[i * L + sb] - muy[i]);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < LP; ++i)
                if (i < L) A.Y[a * L + i] = y[i];
        }
    }
    float part[1] = {e};
    warp_sums<1>(part, A.epart + (int64_t)blockIdx.x * 8);
}

// S_QP per image from the per-warp rows (compensated FP32, FP64 once).
__global__ void __launch_bounds__(1024) k_dcneg_energy(const float *epart, const int *crange, double *out) {
    double e[1];
    image_sums<1>(epart, crange[blockIdx.x], crange[blockIdx.x + 1], e);
    if (threadIdx.x == 0) out[blockIdx.x] = e[0];
}

struct NegSolver {
    cudaStream_t s;
    Scratch sc;
    int L = 0, Lp = 0, batch = 0, storage = 0, nk = 0;
    int64_t n = 0;
    bool potts = true;
    float sumw = 0.f;
    const dcrf_lattice *lats = nullptr;
    float *V[DCRF_MAX_KERNELS] = {};
    void *V1[DCRF_MAX_KERNELS] = {}, *V2[DCRF_MAX_KERNELS] = {}, *tmp[DCRF_MAX_KERNELS] = {};
    float *mu = nullptr, *epart = nullptr;
    int *crange = nullptr;
    Chunk *chunks = nullptr;
    int n_chunks = 0;
    NegArgs A{};

    explicit NegSolver(cudaStream_t st) : s(st), sc(st) {}

    dcrf_status setup(const float *unaries, const dcrf_lattice *lattices, const float *weights, int n_k,
                      const float *compat, int L_, int store, float *Y, int inner, bool need_sumw = true) {
        DCRF_CHECK_STATUS(dcrf_check_lattices(lattices, n_k));
        if (!unaries || !weights || !Y || L_ < 1 || L_ > DCRF_MAX_L || inner < 0) return DCRF_E_INVAL;
        if (store != DCRF_STORAGE_F32 && store != DCRF_STORAGE_F16) return DCRF_E_INVAL;
        lats = lattices;
        nk = n_k;
        L = L_;
        Lp = L <= 8 ? 8 : (L <= 24 ? 24 : 64);
        storage = store;
        n = lattices[0]->n;
        batch = lattices[0]->batch;
        sumw = 0.f;
        for (int m = 0; m < nk; ++m) {
            if (!(weights[m] >= 0.f)) return DCRF_E_INVAL;
            sumw += weights[m];
        }
        if (need_sumw && !(sumw > 0.f)) return DCRF_E_INVAL;
        potts = true;
        std::vector<float> mu_h(L * L);
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j) {
                const float v = compat ? compat[i * L + j] : (i == j ? 0.f : 1.f);
                if (!std::isfinite(v)) return DCRF_E_INVAL;
                mu_h[i * L + j] = v;
                if (v != (i == j ? 0.f : 1.f)) potts = false;
            }
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < i; ++j)
                if (mu_h[i * L + j] != mu_h[j * L + i]) return DCRF_E_INVAL;   // mu must be symmetric
        DCRF_CHECK_STATUS(sc.get(&mu, (size_t)L * L));
        DCRF_TRY(cudaMemcpyAsync(mu, mu_h.data(), L * L * sizeof(float), cudaMemcpyHostToDevice, s));
        const size_t esz = storage == DCRF_STORAGE_F16 ? 2 : 4;
        A.nk = nk;
        for (int m = 0; m < nk; ++m) {
            const dcrf_lattice lat = lattices[m];
            const size_t cnt = (size_t)(lat->m > 0 ? lat->m : 1) * Lp;
            char *b1, *b2, *bt;
            DCRF_CHECK_STATUS(sc.get(&V[m], cnt));
            DCRF_CHECK_STATUS(sc.get(&b1, cnt * esz));
            DCRF_CHECK_STATUS(sc.get(&b2, cnt * esz));
            DCRF_CHECK_STATUS(sc.get(&bt, cnt * esz));
            V1[m] = b1;
            V2[m] = b2;
            tmp[m] = bt;
            A.l[m].pvid = lat->pvid;
            A.l[m].pbary = lat->pbary;
            A.l[m].V1 = b1;
            A.l[m].V2 = b2;
            A.l[m].d1 = lat->d + 1;
            A.l[m].ws0 = (float)(weights[m] * lat->s0);
        }
        auto pc = make_chunks(lattices[0]->point_off, 256);
        n_chunks = (int)pc.size();
        DCRF_CHECK_STATUS(sc.get(&chunks, pc.size() > 0 ? pc.size() : 1));
        if (!pc.empty())
            DCRF_TRY(cudaMemcpyAsync(chunks, pc.data(), pc.size() * sizeof(Chunk), cudaMemcpyHostToDevice, s));
        std::vector<int> cr(batch + 1, 0);
        for (const Chunk &c : pc) cr[c.image + 1] += 8;
        for (int b = 0; b < batch; ++b) cr[b + 1] += cr[b];
        DCRF_CHECK_STATUS(sc.get(&crange, (size_t)batch + 1));
        DCRF_TRY(cudaMemcpyAsync(crange, cr.data(), (batch + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
        DCRF_CHECK_STATUS(sc.get(&epart, (size_t)std::max(1, n_chunks) * 8));
        A.chunks = chunks;
        A.Y = Y;
        A.phi = unaries;
        A.mu = mu;
        A.L = L;
        A.inner = inner;
        A.sumw = sumw;
        A.epart = epart;
        A.status = lattices[0]->status;
        return DCRF_OK;
    }

    // F = (K~ + K~^T) y per lattice (splat once, blur both ways), then the
    // per-pixel pass; energy of the current y into out[batch] (device).
    dcrf_status step(bool update, double *out, bool mf = false) {
        A.mf = mf;
        for (int m = 0; m < nk; ++m) {
            const dcrf_lattice lat = lats[m];
            const size_t cnt = (size_t)(lat->m > 0 ? lat->m : 1) * Lp;
            DCRF_TRY(cudaMemsetAsync(V[m], 0, cnt * sizeof(float), s));
            DCRF_CHECK_STATUS(dcrf_splat_dense(lat, A.Y, L, V[m], Lp, s));
            DCRF_CHECK_STATUS(dcrf_blur(lat, V[m], V1[m], tmp[m], Lp, storage, false, s));
            DCRF_CHECK_STATUS(dcrf_blur(lat, V[m], V2[m], tmp[m], Lp, storage, true, s));
        }
        A.update = update;
        if (n_chunks > 0) {
            ProfScope ps(P_DCNEG_PIXEL, s);
            const bool h = storage == DCRF_STORAGE_F16;
#define DCRF_NEG(LPc) \
    do { \
        if (h) { if (potts) k_dcneg_pixel<LPc, __half, true><<<n_chunks, 256, 0, s>>>(A); \
                 else k_dcneg_pixel<LPc, __half, false><<<n_chunks, 256, 0, s>>>(A); } \
        else { if (potts) k_dcneg_pixel<LPc, float, true><<<n_chunks, 256, 0, s>>>(A); \
               else k_dcneg_pixel<LPc, float, false><<<n_chunks, 256, 0, s>>>(A); } \
    } while (0)
            if (Lp == 8) DCRF_NEG(8);
            else if (Lp == 24) DCRF_NEG(24);
            else DCRF_NEG(64);
#undef DCRF_NEG
            DCRF_LAUNCHED();
        }
        k_dcneg_energy<<<batch, 1024, 0, s>>>(epart, crange, out);
        DCRF_LAUNCHED();
        return DCRF_OK;
    }
};

}  // namespace

extern "C" dcrf_status dcrf_dc_neg(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                   int n_kernels, const float *compat, int L, int outer, int inner, float *Y,
                                   double *qp_energy, int storage, dcrf_stream stream) {
    if (outer < 0 || inner < 0) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    NegSolver S(s);
    DCRF_CHECK_STATUS(S.setup(unaries, lattices, weights, n_kernels, compat, L, storage, Y, inner));
    if (S.n == 0) return DCRF_OK;
    double *qe;
    DCRF_CHECK_STATUS(S.sc.get(&qe, (size_t)(outer + 1) * S.batch));
    for (int t = 0; t <= outer; ++t) DCRF_CHECK_STATUS(S.step(t < outer, qe + (int64_t)t * S.batch));
    if (qp_energy) {
        DCRF_TRY(cudaMemcpyAsync(qp_energy, qe, (size_t)(outer + 1) * S.batch * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
        int h = 0;
        DCRF_TRY(cudaMemcpyAsync(&h, lattices[0]->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DCRF_TRY(cudaStreamSynchronize(s));
        if (h != 0) return (dcrf_status)h;
    }
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_mean_field(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                       int n_kernels, const float *compat, int L, int iters, float *Q,
                                       double *qp_energy, int storage, dcrf_stream stream) {
    if (iters < 0) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    NegSolver S(s);
    DCRF_CHECK_STATUS(S.setup(unaries, lattices, weights, n_kernels, compat, L, storage, Q, 0, false));
    if (S.n == 0) return DCRF_OK;
    double *qe;
    DCRF_CHECK_STATUS(S.sc.get(&qe, (size_t)(iters + 1) * S.batch));
    for (int t = 0; t <= iters; ++t) DCRF_CHECK_STATUS(S.step(t < iters, qe + (int64_t)t * S.batch, true));
    if (qp_energy) {
        DCRF_TRY(cudaMemcpyAsync(qp_energy, qe, (size_t)(iters + 1) * S.batch * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
        int h = 0;
        DCRF_TRY(cudaMemcpyAsync(&h, lattices[0]->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DCRF_TRY(cudaStreamSynchronize(s));
        if (h != 0) return (dcrf_status)h;
    }
    return DCRF_OK;
}

namespace {

// labels[a] = argmax_i Y[a][i] (lowest label on ties); onehot rows if given
__global__ void k_round(const float *__restrict__ Y, int64_t n, int L, int32_t *__restrict__ labels,
                        float *__restrict__ onehot) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    float best = Y[a * L];
    int arg = 0;
    for (int i = 1; i < L; ++i) {
        const float v = Y[a * L + i];
        if (v > best) { best = v; arg = i; }
    }
    labels[a] = arg;
    if (onehot)
        for (int i = 0; i < L; ++i) onehot[a * L + i] = i == arg ? 1.f : 0.f;
}

// Kleinberg-Tardos rounding (end of Section 5): phase t gives label plab[t]
// to every unlabelled pixel whose y of that label exceeds pthr[t].  One thread
// per pixel walks the phases until its first hit; the phase arrays are read by
// every thread of a warp at once (broadcast loads).
__global__ void k_round_kt(const float *__restrict__ Y, int64_t n, int L, const int32_t *__restrict__ plab,
                           const float *__restrict__ pthr, int T, int resume, int32_t *__restrict__ labels,
                           unsigned long long *__restrict__ unassigned) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int x = -1;
    if (a < n) {
        if (resume) x = labels[a] >= 0 ? labels[a] : -1;
        if (x < 0) {
            const float *row = Y + a * L;
            for (int t = 0; t < T; ++t) {
                const int i = __ldg(plab + t);
                if (row[i] > __ldg(pthr + t)) {
                    x = i;
                    break;
                }
            }
        }
        labels[a] = x;
    }
    if (unassigned) {
        const unsigned m = __ballot_sync(0xffffffffu, a < n && x < 0);
        if ((threadIdx.x & 31) == 0 && m) atomicAdd(unassigned, (unsigned long long)__popc(m));
    }
}

__global__ void k_onehot(const int32_t *__restrict__ labels, int64_t n, int L, float *__restrict__ Y,
                         int *__restrict__ status) {
    const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int x = labels[a];
    if (x < 0 || x >= L) dcrf_flag(status, DCRF_E_INVAL);
    for (int i = 0; i < L; ++i) Y[a * L + i] = i == x ? 1.f : 0.f;
}

}  // namespace

extern "C" dcrf_status dcrf_round(const float *Y, int64_t n, int L, int32_t *labels, float *onehot,
                                  dcrf_stream stream) {
    if (n < 0 || L < 1 || (n > 0 && (!Y || !labels))) return DCRF_E_INVAL;
    if (n == 0) return DCRF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_round<<<nblocks(n, 256), 256, 0, s>>>(Y, n, L, labels, onehot);
    DCRF_LAUNCHED();
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_round_kt(const float *Y, int64_t n, int L, int n_phases, const int32_t *phase_labels,
                                     const float *phase_thresholds, int resume, int32_t *labels,
                                     int64_t *unassigned, dcrf_stream stream) {
    if (n < 0 || L < 1 || n_phases < 0 || (n > 0 && (!Y || !labels)) ||
        (n_phases > 0 && (!phase_labels || !phase_thresholds)))
        return DCRF_E_INVAL;
    for (int t = 0; t < n_phases; ++t)
        if (phase_labels[t] < 0 || phase_labels[t] >= L || !(phase_thresholds[t] >= 0.f) ||
            !(phase_thresholds[t] < 1.f))
            return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        if (unassigned) *unassigned = 0;
        return DCRF_OK;
    }
    Scratch sc(s);
    int32_t *plab = nullptr;
    float *pthr = nullptr;
    unsigned long long *cnt = nullptr;
    const int T = n_phases;
    DCRF_CHECK_STATUS(sc.get(&plab, (size_t)(T > 0 ? T : 1)));
    DCRF_CHECK_STATUS(sc.get(&pthr, (size_t)(T > 0 ? T : 1)));
    if (T > 0) {
        DCRF_TRY(cudaMemcpyAsync(plab, phase_labels, T * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        DCRF_TRY(cudaMemcpyAsync(pthr, phase_thresholds, T * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    if (unassigned) {
        DCRF_CHECK_STATUS(sc.get(&cnt, 1));
        DCRF_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    }
    k_round_kt<<<nblocks(n, 256), 256, 0, s>>>(Y, n, L, plab, pthr, T, resume, labels, cnt);
    DCRF_LAUNCHED();
    if (unassigned) {
        unsigned long long h = 0;
        DCRF_TRY(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
        DCRF_TRY(cudaStreamSynchronize(s));
        *unassigned = (int64_t)h;
    }
    return DCRF_OK;
}

extern "C" dcrf_status dcrf_labelling_energy(const float *unaries, const dcrf_lattice *lattices,
                                             const float *weights, int n_kernels, const float *compat, int L,
                                             const int32_t *labels, double *energy, int storage,
                                             dcrf_stream stream) {
    if (!energy || !labels) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    DCRF_CHECK_STATUS(dcrf_check_lattices(lattices, n_kernels));
    const int64_t n = lattices[0]->n;
    Scratch sc(s);
    float *Y;
    DCRF_CHECK_STATUS(sc.get(&Y, (size_t)(n > 0 ? n : 1) * (L > 0 ? L : 1)));
    NegSolver S(s);
    DCRF_CHECK_STATUS(S.setup(unaries, lattices, weights, n_kernels, compat, L, storage, Y, 0, false));
    if (n > 0) {
        k_onehot<<<nblocks(n, 256), 256, 0, s>>>(labels, n, L, Y, S.A.status);
        DCRF_LAUNCHED();
    }
    double *qe;
    DCRF_CHECK_STATUS(S.sc.get(&qe, (size_t)S.batch));
    if (n > 0) DCRF_CHECK_STATUS(S.step(false, qe));
    else DCRF_TRY(cudaMemsetAsync(qe, 0, S.batch * sizeof(double), s));
    DCRF_TRY(cudaMemcpyAsync(energy, qe, S.batch * sizeof(double), cudaMemcpyDeviceToHost, s));
    int h = 0;
    DCRF_TRY(cudaMemcpyAsync(&h, lattices[0]->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    DCRF_TRY(cudaStreamSynchronize(s));
    if (h != 0) return (dcrf_status)h;
    return DCRF_OK;
}

// ---------------------------------------------------------------------------
// Reverse mode through unrolled Frank-Wolfe.
//
// With P = Op(y) = (Psi + D) y, one iteration is y+ = y + alpha (s - y) with
// alpha = -B / (2A) when A > 0 and 0 < alpha < 1 (else alpha is locally
// constant), s piecewise constant.  With Delta = s - y and
// u = y + (2 alpha - 1) Delta:
//   d alpha / d y   = (lin + Op u + Op^T u) / (2A),   d alpha / d phi = -Delta / (2A),
//   d alpha / d w_m = -(dB_m + 2 alpha dA_m) / (2A),  dA_m = <Delta, Op_m' Delta>,
//   dB_m = -<d_m', Delta> + <y, Op_m' Delta> + <Delta, Op_m' y>,
// Op_m' v = mu (K~_m v - v) + d_m' o v,  d_m' = (sum_j |mu_ij|) (K~_m 1 - 1) [c > 0].
// Reverse step: abar = <ybar, Delta>, ybar <- (1 - alpha) ybar + abar d alpha/dy.
namespace {

constexpr int NB = 1 + 2 * DCRF_MAX_KERNELS;   // abar, dA_m, dB_m

struct BwArgs {
    const Chunk *chunks;
    const float *Yt;                  // [n][L] y^t
    const uint8_t *st;                // [n] s^t
    const float *lin;                 // [n][L] phi - d
    const float *c;                   // [n] clamped c
    const float *ones[DCRF_MAX_KERNELS];
    const float *KY[DCRF_MAX_KERNELS];
    const float *KS[DCRF_MAX_KERNELS];
    const float *KTu[DCRF_MAX_KERNELS];
    float w[DCRF_MAX_KERNELS];
    int nk;
    const float *mu;
    const float *musum;
    float sumw;
    int L;
    float *ybar;
    float *phibar;
    double *acc;                      // [batch][NB]
    const float *coef;                // [batch] abar / (2A) when interior, else 0
    const float *oma;                 // [batch] 1 - alpha
    const float *tam1;                // [batch] 2 alpha - 1
};

template <int LP, bool POTTS>
__device__ __forceinline__ void apply_mu(const float (&x)[LP], float (&out)[LP], const float *mu, int L, bool transpose) {
    if (POTTS) {
        float tot = 0.f;
#pragma unroll
        for (int i = 0; i < LP; ++i) tot += i < L ? x[i] : 0.f;
#pragma unroll
        for (int i = 0; i < LP; ++i) out[i] = i < L ? tot - x[i] : 0.f;
    } else {
#pragma unroll
        for (int i = 0; i < LP; ++i) {
            float acc = 0.f;
#pragma unroll 8
            for (int j = 0; j < LP; ++j)
                if (i < L && j < L) acc += (transpose ? mu[j * L + i] : mu[i * L + j]) * x[j];
            out[i] = acc;
        }
    }
}

__device__ __forceinline__ float active_c(const BwArgs &B, int64_t a) {
    float s = 0.f, sw = 0.f;
    for (int m = 0; m < B.nk; ++m) { s += B.w[m] * B.ones[m][a]; sw += B.w[m]; }
    return s - sw > 0.f ? 1.f : 0.f;
}

template <int LP, bool POTTS>
__global__ void __launch_bounds__(128) k_bw_reduce(BwArgs B) {
    const Chunk ch = B.chunks[blockIdx.x];
    double part[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) part[q] = 0.0;
    if ((int)threadIdx.x < ch.count) {
        const int64_t a = ch.begin + threadIdx.x;
        const int L = B.L;
        const int s = B.st[a];
        float y[LP], dl[LP];
        float ab = 0.f;
#pragma unroll
        for (int i = 0; i < LP; ++i) {
            y[i] = i < L ? B.Yt[a * L + i] : 0.f;
            dl[i] = i < L ? (i == s ? 1.f : 0.f) - y[i] : 0.f;
            if (i < L) ab += B.ybar[a * L + i] * dl[i];
        }
        part[0] = ab;
        const float act = active_c(B, a);
        for (int m = 0; m < B.nk; ++m) {
            float xd[LP], xy[LP], md[LP], my[LP];
            const float dm = (B.ones[m][a] - 1.f) * act;
#pragma unroll
            for (int i = 0; i < LP; ++i) {
                const float ky = i < L ? B.KY[m][a * L + i] : 0.f;
                const float ks = i < L ? B.KS[m][a * L + i] : 0.f;
                xd[i] = (ks - ky) - dl[i];
                xy[i] = ky - y[i];
            }
            apply_mu<LP, POTTS>(xd, md, B.mu, L, false);
            apply_mu<LP, POTTS>(xy, my, B.mu, L, false);
            float dA = 0.f, dB = 0.f;
#pragma unroll
            for (int i = 0; i < LP; ++i) {
                if (i < L) {
                    const float ddi = (POTTS ? (float)(L - 1) : B.musum[i]) * dm;
                    const float opd = md[i] + ddi * dl[i];     // Op_m' Delta
                    const float opy = my[i] + ddi * y[i];      // Op_m' y
                    dA += dl[i] * opd;
                    dB += -ddi * dl[i] + y[i] * opd + dl[i] * opy;
                }
            }
            part[1 + 2 * m] = dA;
            part[2 + 2 * m] = dB;
        }
    }
    block_reduce_add<NB>(part, B.acc + (int64_t)ch.image * NB);
}

__global__ void k_bw_coef(int batch, int nk, double *acc, const dcrf_fw_record *rec, int t, float *coef,
                          float *oma, float *tam1, double *wbar) {
    if (threadIdx.x != 0) return;
    for (int b = 0; b < batch; ++b) {
        const dcrf_fw_record r = rec[(int64_t)t * batch + b];
        double *g = acc + (int64_t)b * NB;
        const bool interior = r.A > 0.0 && r.alpha > 0.0 && r.alpha < 1.0;
        const double abar = g[0];
        coef[b] = interior ? (float)(abar / (2.0 * r.A)) : 0.f;
        oma[b] = (float)(1.0 - r.alpha);
        tam1[b] = (float)(2.0 * r.alpha - 1.0);
        if (interior)
            for (int m = 0; m < nk; ++m)
                wbar[m] += abar * (-(g[2 + 2 * m] + 2.0 * r.alpha * g[1 + 2 * m]) / (2.0 * r.A));
        for (int q = 0; q < NB; ++q) g[q] = 0.0;
    }
}

__global__ void k_bw_dense(const Chunk *chunks, const float *Yt, const uint8_t *st, int L, const float *tam1,
                           float *S, float *U) {
    const Chunk ch = chunks[blockIdx.x];
    if ((int)threadIdx.x >= ch.count) return;
    const int64_t a = ch.begin + threadIdx.x;
    const int s = st[a];
    const float k = tam1[ch.image];
    for (int i = 0; i < L; ++i) {
        const float y = Yt[a * L + i];
        const float e = i == s ? 1.f : 0.f;
        S[a * L + i] = e;
        U[a * L + i] = y + k * (e - y);      // u = y + (2 alpha - 1)(s - y)
    }
}

template <int LP, bool POTTS>
__global__ void __launch_bounds__(128) k_bw_update(BwArgs B) {
    const Chunk ch = B.chunks[blockIdx.x];
    if ((int)threadIdx.x >= ch.count) return;
    const int64_t a = ch.begin + threadIdx.x;
    const int L = B.L;
    const int s = B.st[a];
    const float cf = B.coef[ch.image], om = B.oma[ch.image], k = B.tam1[ch.image];
    const float ca = B.c[a];
    float y[LP], dl[LP], xy[LP], xd[LP], xu[LP];
#pragma unroll
    for (int i = 0; i < LP; ++i) {
        y[i] = i < L ? B.Yt[a * L + i] : 0.f;
        dl[i] = i < L ? (i == s ? 1.f : 0.f) - y[i] : 0.f;
        xy[i] = -B.sumw * y[i];
        xd[i] = -B.sumw * dl[i];
        xu[i] = -B.sumw * (y[i] + k * dl[i]);
    }
    for (int m = 0; m < B.nk; ++m) {
#pragma unroll
        for (int i = 0; i < LP; ++i) {
            if (i < L) {
                const float ky = B.KY[m][a * L + i], ks = B.KS[m][a * L + i], kt = B.KTu[m][a * L + i];
                xy[i] += B.w[m] * ky;
                xd[i] += B.w[m] * (ks - ky);
                xu[i] += B.w[m] * kt;
            }
        }
    }
    float my[LP], md[LP], mu_[LP];
    apply_mu<LP, POTTS>(xy, my, B.mu, L, false);
    apply_mu<LP, POTTS>(xd, md, B.mu, L, false);
    apply_mu<LP, POTTS>(xu, mu_, B.mu, L, true);
#pragma unroll
    for (int i = 0; i < LP; ++i) {
        if (i < L) {
            const float di = (POTTS ? (float)(L - 1) : B.musum[i]) * ca;
            const float u = y[i] + k * dl[i];
            const float opy = my[i] + di * y[i];
            const float opd = md[i] + di * dl[i];
            const float opu = opy + k * opd;
            const float optu = mu_[i] + di * u;
            const float g = B.ybar[a * L + i];
            B.ybar[a * L + i] = om * g + cf * (B.lin[a * L + i] + opu + optu);
            B.phibar[a * L + i] -= cf * dl[i];
        }
    }
}

template <int LP, bool POTTS>
dcrf_status bw_launch(BwArgs &B, int nchunks, bool reduce, cudaStream_t s) {
    if (nchunks == 0) return DCRF_OK;
    if (reduce) k_bw_reduce<LP, POTTS><<<nchunks, 128, 0, s>>>(B);
    else k_bw_update<LP, POTTS><<<nchunks, 128, 0, s>>>(B);
    DCRF_LAUNCHED();
    return DCRF_OK;
}

dcrf_status bw_dispatch(BwArgs &B, int Lp, bool potts, int nchunks, bool reduce, cudaStream_t s) {
    if (Lp == 8) return potts ? bw_launch<8, true>(B, nchunks, reduce, s) : bw_launch<8, false>(B, nchunks, reduce, s);
    if (Lp == 24) return potts ? bw_launch<24, true>(B, nchunks, reduce, s) : bw_launch<24, false>(B, nchunks, reduce, s);
    return potts ? bw_launch<64, true>(B, nchunks, reduce, s) : bw_launch<64, false>(B, nchunks, reduce, s);
}

// out = K~ in (or K~^T in) for one lattice, float32 values.
dcrf_status dense_filter(const dcrf_lattice lat, const float *in, int L, int Lp, float *out, bool adjoint,
                         float *V, float *dst, float *tmp, cudaStream_t s) {
    if (lat->n == 0) return DCRF_OK;
    DCRF_TRY(cudaMemsetAsync(V, 0, (size_t)lat->m * Lp * sizeof(float), s));
    DCRF_CHECK_STATUS(dcrf_splat_dense(lat, in, L, V, Lp, s));
    DCRF_CHECK_STATUS(dcrf_blur(lat, V, dst, tmp, Lp, DCRF_STORAGE_F32, adjoint, s));
    return dcrf_slice_f32(lat, dst, Lp, L, out, s);
}

}  // namespace

extern "C" dcrf_status dcrf_qp_fw_backward(const float *unaries, const dcrf_lattice *lattices, const float *weights,
                                           int n_kernels, const float *compat, int L, int iters, const float *Y0,
                                           const float *dYT, float *dphi, float *dY0, double *dweights,
                                           uint8_t *s_tape, dcrf_stream stream) {
    if (iters < 0 || !Y0 || !dYT || !dphi) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Solver S(s);
    float *Y;
    DCRF_CHECK_STATUS(dcrf_check_lattices(lattices, n_kernels));
    const int64_t n = lattices[0]->n;
    if (L < 1 || L > DCRF_MAX_L) return DCRF_E_INVAL;
    DCRF_CHECK_STATUS(S.sc.get(&Y, (size_t)(n > 0 ? n : 1) * L));
    if (n > 0) DCRF_TRY(cudaMemcpyAsync(Y, Y0, n * L * sizeof(float), cudaMemcpyDeviceToDevice, s));
    DCRF_CHECK_STATUS(S.setup(unaries, lattices, weights, n_kernels, compat, L, DCRF_STORAGE_F32, Y, iters));
    const int nk = S.nk, Lp = S.Lp, batch = S.batch;
    double *wbar;
    DCRF_CHECK_STATUS(S.sc.get(&wbar, (size_t)nk));
    DCRF_TRY(cudaMemsetAsync(wbar, 0, nk * sizeof(double), s));
    if (n > 0) DCRF_TRY(cudaMemsetAsync(dphi, 0, n * L * sizeof(float), s));
    if (n == 0) {
        if (dweights) for (int m = 0; m < nk; ++m) dweights[m] = 0.0;
        return DCRF_OK;
    }
    // forward recompute with a checkpoint of (y^t, s^t) before every iteration
    float *ytape;
    uint8_t *stape;
    DCRF_CHECK_STATUS(S.sc.get(&ytape, (size_t)(iters > 0 ? iters : 1) * n * L));
    DCRF_CHECK_STATUS(S.sc.get(&stape, (size_t)(iters > 0 ? iters : 1) * n));
    DCRF_CHECK_STATUS(S.pixel(Y, nullptr, true));
    for (int t = 0; t < iters; ++t) {
        DCRF_TRY(cudaMemcpyAsync(ytape + (int64_t)t * n * L, Y, n * L * sizeof(float), cudaMemcpyDeviceToDevice, s));
        DCRF_TRY(cudaMemcpyAsync(stape + (int64_t)t * n, S.sidx, n, cudaMemcpyDeviceToDevice, s));
        DCRF_CHECK_STATUS(S.iterate(Y, nullptr));
    }
    // reverse sweep
    float *ybar, *Sd, *U, *KY[DCRF_MAX_KERNELS], *KS[DCRF_MAX_KERNELS], *KTu[DCRF_MAX_KERNELS];
    float *coef, *oma, *tam1, *V, *dst, *tmp;
    double *acc;
    const size_t nl = (size_t)n * L;
    DCRF_CHECK_STATUS(S.sc.get(&ybar, nl));
    DCRF_CHECK_STATUS(S.sc.get(&Sd, nl));
    DCRF_CHECK_STATUS(S.sc.get(&U, nl));
    int64_t mmax = 1;
    for (int m = 0; m < nk; ++m) {
        DCRF_CHECK_STATUS(S.sc.get(&KY[m], nl));
        DCRF_CHECK_STATUS(S.sc.get(&KS[m], nl));
        DCRF_CHECK_STATUS(S.sc.get(&KTu[m], nl));
        mmax = std::max<int64_t>(mmax, lattices[m]->m);
    }
    DCRF_CHECK_STATUS(S.sc.get(&V, (size_t)mmax * Lp));
    DCRF_CHECK_STATUS(S.sc.get(&dst, (size_t)mmax * Lp));
    DCRF_CHECK_STATUS(S.sc.get(&tmp, (size_t)mmax * Lp));
    DCRF_CHECK_STATUS(S.sc.get(&coef, (size_t)batch));
    DCRF_CHECK_STATUS(S.sc.get(&oma, (size_t)batch));
    DCRF_CHECK_STATUS(S.sc.get(&tam1, (size_t)batch));
    DCRF_CHECK_STATUS(S.sc.get(&acc, (size_t)batch * NB));
    DCRF_TRY(cudaMemsetAsync(acc, 0, batch * NB * sizeof(double), s));
    DCRF_TRY(cudaMemsetAsync(tam1, 0, batch * sizeof(float), s));
    DCRF_TRY(cudaMemcpyAsync(ybar, dYT, nl * sizeof(float), cudaMemcpyDeviceToDevice, s));
    // 128-row chunks for the reverse kernels
    auto ch = make_chunks(lattices[0]->point_off, 128);
    Chunk *chd;
    DCRF_CHECK_STATUS(S.sc.get(&chd, ch.size() > 0 ? ch.size() : 1));
    DCRF_TRY(cudaMemcpyAsync(chd, ch.data(), ch.size() * sizeof(Chunk), cudaMemcpyHostToDevice, s));
    const int nch = (int)ch.size();
    BwArgs B{};
    B.chunks = chd;
    B.lin = S.lin;
    B.c = S.c;
    B.nk = nk;
    for (int m = 0; m < nk; ++m) {
        B.ones[m] = lattices[m]->ones;
        B.KY[m] = KY[m];
        B.KS[m] = KS[m];
        B.KTu[m] = KTu[m];
        B.w[m] = weights[m];
    }
    B.mu = S.mu;
    B.musum = S.musum;
    B.sumw = S.sumw;
    B.L = L;
    B.ybar = ybar;
    B.phibar = dphi;
    B.acc = acc;
    B.coef = coef;
    B.oma = oma;
    B.tam1 = tam1;
    for (int t = iters - 1; t >= 0; --t) {
        const float *Yt = ytape + (int64_t)t * n * L;
        const uint8_t *st = stape + (int64_t)t * n;
        B.Yt = Yt;
        B.st = st;
        k_bw_dense<<<nch, 128, 0, s>>>(chd, Yt, st, L, tam1, Sd, U);   // S only (U recomputed below)
        DCRF_LAUNCHED();
        for (int m = 0; m < nk; ++m) {
            DCRF_CHECK_STATUS(dense_filter(lattices[m], Yt, L, Lp, KY[m], false, V, dst, tmp, s));
            DCRF_CHECK_STATUS(dense_filter(lattices[m], Sd, L, Lp, KS[m], false, V, dst, tmp, s));
        }
        DCRF_CHECK_STATUS(bw_dispatch(B, Lp, S.potts, nch, true, s));
        k_bw_coef<<<1, 32, 0, s>>>(batch, nk, acc, S.rec, t, coef, oma, tam1, wbar);
        DCRF_LAUNCHED();
        k_bw_dense<<<nch, 128, 0, s>>>(chd, Yt, st, L, tam1, Sd, U);   // u with this iteration's alpha
        DCRF_LAUNCHED();
        for (int m = 0; m < nk; ++m)
            DCRF_CHECK_STATUS(dense_filter(lattices[m], U, L, Lp, KTu[m], true, V, dst, tmp, s));
        DCRF_CHECK_STATUS(bw_dispatch(B, Lp, S.potts, nch, false, s));
    }
    if (dY0) DCRF_TRY(cudaMemcpyAsync(dY0, ybar, nl * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (s_tape && iters > 0)
        DCRF_TRY(cudaMemcpyAsync(s_tape, stape, (size_t)iters * n, cudaMemcpyDeviceToDevice, s));
    if (dweights) {
        DCRF_TRY(cudaMemcpyAsync(dweights, wbar, nk * sizeof(double), cudaMemcpyDeviceToHost, s));
        int h = 0;
        DCRF_TRY(cudaMemcpyAsync(&h, S.status, sizeof(int), cudaMemcpyDeviceToHost, s));
        DCRF_TRY(cudaStreamSynchronize(s));
        if (h != 0) return (dcrf_status)h;
    }
    return DCRF_OK;
}
