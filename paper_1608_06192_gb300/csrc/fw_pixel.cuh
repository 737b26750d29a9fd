// Pixel pass of the Frank-Wolfe solver (Algorithm 1, Appendix B): the layouts
// of the per-iteration pixel kernel, its arguments and the per-warp sums.
// Included once, by fw.cu (the solver that launches it).
#pragma once

#include "common.cuh"

namespace {

// Pixel-kernel variants (pixels per block = threads, minimum blocks per SM);
// the autotuner picks one per (labels, storage, compatibility, size) at first use.
// Pixel-kernel modes: kFix gathers the corner rows of the common two-kernel
// case (bilateral d = 5, spatial d = 2) with every index loaded up front;
// kF2 accumulates the gathered rows with packed two-wide FP32 FMAs.  (A
// shared-memory hash aggregation of the splat was measured 2x slower than
// plain FP32 reductions in L2: many pixels of a block hit the same key.)
// kL3 is the label-split layout (three lanes per pixel, 80 pixels per block,
// see pixel3); kEarly gathers the corner rows while the chunk's y and lin
// rows are still in flight to shared memory.
// kBulk moves the chunk's y and lin rows in and y' out with bulk (TMA) copies
// completed on an mbarrier, where the rows are 16-byte aligned.
// kLean (Potts) computes y' and the label totals in one pass and tracks only
// the argmin, its gradient and X(s') in the label loop.
// kL21 fixes L = 21 at compile time (the label count of the segmentation
// workloads): the loops over the padded 24 labels lose their runtime bounds
// and the padding labels' accumulators and FMAs go away.
constexpr int kFix = 1, kF2 = 2, kL3 = 4, kEarly = 8, kBulk = 16, kLean = 32, kL21 = 64;
constexpr int kPixVariants = 19;
constexpr int kPixPB[kPixVariants] = {256, 128, 256, 128, 256, 80, 128, 256, 128, 128,
                                      128, 128, 128, 128, 128, 128, 128, 128, 128};
constexpr int kPixMB[kPixVariants] = {4, 8, 3, 6, 3, 0, 6, 3, 6, 8, 7, 8, 7, 6, 7, 8, 7, 8, 6};
constexpr int kPixMode[kPixVariants] = {0,           0,           kFix,         kFix,
                                        kFix | kF2,  kL3,         kFix | kEarly, kFix | kEarly,
                                        kFix | kF2 | kEarly, kFix | kEarly, kFix | kF2 | kEarly,
                                        kFix | kF2 | kEarly, kFix | kF2 | kEarly | kBulk,
                                        kFix | kF2 | kEarly | kBulk, kFix | kF2 | kEarly | kBulk | kLean,
                                        kFix | kF2 | kEarly | kBulk | kLean,
                                        kFix | kF2 | kEarly | kBulk | kLean | kL21,
                                        kFix | kF2 | kEarly | kBulk | kLean | kL21,
                                        kFix | kF2 | kEarly | kBulk | kLean | kL21};
// whether variant v can run a problem with L labels
constexpr bool pixel_variant_fits(int v, int L) { return (kPixMode[v] & kL21) == 0 || L == 21; }
// chunk list of a pixel-block size (256, 128 or 80 pixels)
constexpr int chunk_list(int pb) { return pb == 256 ? 0 : (pb == 128 ? 1 : 2); }
constexpr int chunk_warps(int list) { return list == 0 ? 8 : (list == 1 ? 4 : 8); }
constexpr int kVertBlock = 128;  // vertices per block
constexpr int NS = 8;            // per-pixel scalar sums, see k_fw_pixel

struct FwLat {
    const int32_t *pvid;
    const float *pbary;
    const int32_t *vimg;
    int64_t m;
    int d1;
    float ws0;       // w_m * s0_m
    float *Ylat;     // [m][Lp] S y
    float *BY;       // [m][Lp] B S y (float32 master)
    __half *BYh;     // [m][Lp] half copy of BY sliced by the pixel kernel (half storage only)
    // One-hot splats in fixed point (value = entry * qs[1]; integer sums, so
    // deterministic), two buffers used in turn: at iteration t, Sq holds
    // S s^t (read by the blur and the line search) and Sp holds S s^{t-1},
    // which the line-search kernel folds into Ylat and clears; the pixel
    // pass then splats s^{t+1} into St (= Sp; = Sq in the start pass).
    uint32_t *Sq;
    uint32_t *Sp;
    uint32_t *St;
    const float *qs; // {2^k, 2^-k} of this lattice's fixed point
    void *BS;        // [m][Lp] B S s (float or half)
    void *tmp;       // blur scratch (same type as BS)
};

struct FwLats {
    FwLat l[DCRF_MAX_KERNELS];
    int nk;
};

__device__ __forceinline__ float4 ld4(const float *p, int64_t i) { return reinterpret_cast<const float4 *>(p)[i]; }
__device__ __forceinline__ float4 ld4(const __half *p, int64_t i) {
    uint2 raw = reinterpret_cast<const uint2 *>(p)[i];
    float2 a = __half22float2(*reinterpret_cast<__half2 *>(&raw.x));
    float2 b = __half22float2(*reinterpret_cast<__half2 *>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 ld4q(const uint32_t *p, int64_t i, float inv) {
    const uint4 u = reinterpret_cast<const uint4 *>(p)[i];
    return make_float4((float)u.x * inv, (float)u.y * inv, (float)u.z * inv, (float)u.w * inv);
}
__device__ __forceinline__ void st4(float *p, int64_t i, float4 v) { reinterpret_cast<float4 *>(p)[i] = v; }
__device__ __forceinline__ void st4h(__half *p, int64_t i, float4 v) {
    __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<uint32_t *>(&lo);
    raw.y = *reinterpret_cast<uint32_t *>(&hi);
    reinterpret_cast<uint2 *>(p)[i] = raw;
}

template <int N>
__device__ __forceinline__ void block_reduce_add(double (&v)[N], double *acc) {
    __shared__ double red[32][N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][q] = x;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            double x = lane < nw ? red[lane][q] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) atomicAdd(acc + q, x);
        }
    }
}

// Pixel phase of one iteration (or the start, alpha == 0).  It runs after the
// lattice update, so BY already holds B S y' for y' = y + alpha (s - y):
//   y'   = y + alpha (onehot(s) - y)
//   Ky'  = sum_m w_m s0_m sum_k b_k BY_m[v_k]
//   P    = mu (Ky' - sum_w y') + d o y'         = (Psi + D) y'
//   g    = lin + 2 P,  s' = argmin_i g_i (lowest index on ties)
// Sums per image (FP64), at y' and s':
//   0: <lin, y'>   1: <y', P>   2: lin(s')   3: P(s')
//   4: -sum_w <y', mu e_s'> + y'(s') d(s')   (pixel part of <y', (Psi+D) s'>)
//   5: -sum_w mu(s', s') + d(s')            (pixel part of <s', (Psi+D) s'>)
//   6: <y', D y'>  7: <phi, y'> (only when phi is given)
// and S s' is splatted into Sq: every corner adds its barycentric weight
// rounded to a multiple of 2^-k (integer reductions in L2, so the sums and
// everything after them do not depend on the order of the atomics).
struct PixArgs {
    const Chunk *chunks;
    const double *alpha;   // [batch] or null (start: alpha = 0)
    float *Y;              // [n][L]
    const float *lin;      // [n][L] linear term (phi - d, or the CCCP one)
    const float *phi;      // [n][L] or null
    uint8_t *s;            // [n]
    const float *c;        // [n] c_a >= 0
    const float *mu;       // [L][L] (general mu only)
    const float *musum;    // [L]
    float sumw;
    int L;
    int Ls;                // shared-memory row stride (odd)
    bool y16;              // Y starts on a 16-byte boundary (lin always does)
    float *cpart;          // [chunks][PB / 32][NS] per-warp sums
    int *status;
};

template <typename TB>
__device__ __forceinline__ const TB *slice_src(const FwLat &lt);
template <>
__device__ __forceinline__ const float *slice_src<float>(const FwLat &lt) { return lt.BY; }
template <>
__device__ __forceinline__ const __half *slice_src<__half>(const FwLat &lt) { return lt.BYh; }

// Eight labels of a lattice row: 2 x float4 (float32) or 1 x uint4 (half).
__device__ __forceinline__ void ld8(const float *p, int64_t row, int LP, int h, float (&o)[8]) {
    const float4 *q = reinterpret_cast<const float4 *>(p + row * LP + 8 * h);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void ld8(const __half *p, int64_t row, int LP, int h, float (&o)[8]) {
    const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(p + row * LP + 8 * h));
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
    const float2 c = __half22float2(*reinterpret_cast<const __half2 *>(&raw.z));
    const float2 d = __half22float2(*reinterpret_cast<const __half2 *>(&raw.w));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y; o[4] = c.x; o[5] = c.y; o[6] = d.x; o[7] = d.y;
}

// s + e = a + b exactly (Knuth's two-sum; no FMA contraction applies).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// (hi, lo) += (h2, l2) with the rounding error of hi + h2 kept in lo.
__device__ __forceinline__ void add_comp(float &hi, float &lo, float h2, float l2) {
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo += l2 + e;
}

// Per-warp FP32 sums of N values: lane 0 of warp w stores them to
// out[w N .. w N + N) (one row of per-warp partials, summed across rows in
// compensated FP32 by the step kernel).  No block barrier and no FP64 here.
template <int N>
__device__ __forceinline__ void warp_sums(float (&v)[N], float *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        float x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) out[warp * N + q] = x;
    }
}

__device__ __forceinline__ void cp_async4(float *sdst, const float *gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(float *sdst, const float *gsrc) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Bulk (TMA) copies between global and shared memory with an mbarrier.
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared, completion counted on bar (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
constexpr long long kWaitPolls = 1ll << 22;        // first bounded wait of a tile copy
constexpr long long kWaitPollsLast = 1ll << 26;    // the second one, after DCRF_E_TIMEOUT was flagged
// Waits for phase 0 of bar with a bounded number of polls; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, long long polls = kWaitPolls) {
    for (long long i = 0; i < polls; ++i) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_addr(bar)) : "memory");
        if (done) return true;
    }
    return false;
}
// shared -> global bulk store of this thread; returns after the shared source was read
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Whether the chunk's y and lin rows can move as two bulk copies: dense rows,
// 16-byte aligned start and size on both sides.
__device__ __forceinline__ bool tile_bulk_ok(const PixArgs &A, const Chunk &ch) {
    const int64_t base = ch.begin * (int64_t)A.L;
    const int64_t cnt = ch.count * (int64_t)A.L;
    return A.y16 && A.Ls == A.L && ((base | cnt) & 3) == 0 && cnt > 0;
}

// Issues the asynchronous copies of one chunk's y and lin rows into shared
// memory (row stride Ls); the (row, column) of element i advance incrementally.
__device__ __forceinline__ void tile_load_async(const PixArgs &A, const Chunk &ch, float *sy, float *sl) {
    const int L = A.L;
    const int64_t base = ch.begin * (int64_t)L;
    const int cnt = ch.count * L;
    if (A.y16 && A.Ls == L && ((base | cnt) & 3) == 0) {
        // dense rows, 16-byte aligned on both sides (Y, lin are 16-byte
        // aligned allocations and sy, sl start on 16-byte shared offsets)
        for (int i = 4 * threadIdx.x; i < cnt; i += 4 * blockDim.x) {
            cp_async16(sy + i, A.Y + base + i);
            cp_async16(sl + i, A.lin + base + i);
        }
    } else if (A.Ls == L) {
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            cp_async4(sy + i, A.Y + base + i);
            cp_async4(sl + i, A.lin + base + i);
        }
    } else {
        int r = threadIdx.x / L, c = threadIdx.x - r * L;
        const int dr = blockDim.x / L, dc = blockDim.x - dr * L;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            cp_async4(sy + r * A.Ls + c, A.Y + base + i);
            cp_async4(sl + r * A.Ls + c, A.lin + base + i);
            r += dr;
            c += dc;
            if (c >= L) { c -= L; ++r; }
        }
    }
}

__device__ __forceinline__ void tile_store(const PixArgs &A, const Chunk &ch, const float *sy) {
    const int L = A.L;
    const int64_t base = ch.begin * (int64_t)L;
    const int cnt = ch.count * L;
    if (A.y16 && A.Ls == L && ((base | cnt) & 3) == 0) {
        for (int i = 4 * threadIdx.x; i < cnt; i += 4 * blockDim.x)
            *reinterpret_cast<float4 *>(A.Y + base + i) = *reinterpret_cast<const float4 *>(sy + i);
    } else if (A.Ls == L) {
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) A.Y[base + i] = sy[i];
    } else {
        int r = threadIdx.x / L, c = threadIdx.x - r * L;
        const int dr = blockDim.x / L, dc = blockDim.x - dr * L;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            A.Y[base + i] = sy[r * A.Ls + c];
            r += dr;
            c += dc;
            if (c >= L) { c -= L; ++r; }
        }
    }
}

// acc[8h .. 8h+7] += w o[0 .. 7], as scalar or packed FMAs (same rounding)
template <int LP, bool F2>
__device__ __forceinline__ void acc8(float (&acc)[LP], int h, float w, const float (&o)[8]) {
    if constexpr (F2) {
        const float2 w2 = make_float2(w, w);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 r = __ffma2_rn(w2, make_float2(o[2 * j], o[2 * j + 1]),
                                        make_float2(acc[8 * h + 2 * j], acc[8 * h + 2 * j + 1]));
            acc[8 * h + 2 * j] = r.x;
            acc[8 * h + 2 * j + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[8 * h + j] += w * o[j];
    }
}

// K~ y' for the two-kernel case with d+1 = DA and DB corners: every vertex id
// and weight is loaded first, then every corner row, so that the dependent
// loads of one pixel overlap (an absent corner reads row 0 with weight 0).
template <int LP, typename TB, int DA, int DB, bool F2>
__device__ __forceinline__ void gather_pair(const FwLat &la, const FwLat &lb, int64_t a, float (&ky)[LP]) {
    int v[DA + DB];
    float w[DA + DB];
#pragma unroll
    for (int k = 0; k < DA; ++k) {
        v[k] = __ldg(la.pvid + a * DA + k);
        w[k] = __ldg(la.pbary + a * DA + k) * la.ws0;
    }
#pragma unroll
    for (int k = 0; k < DB; ++k) {
        v[DA + k] = __ldg(lb.pvid + a * DB + k);
        w[DA + k] = __ldg(lb.pbary + a * DB + k) * lb.ws0;
    }
    const TB *sa = slice_src<TB>(la), *sb = slice_src<TB>(lb);
#pragma unroll
    for (int k = 0; k < DA + DB; ++k) {
        const int vk = v[k] < 0 ? 0 : v[k];
        const float wk = v[k] < 0 ? 0.f : w[k];
#pragma unroll
        for (int h = 0; h < LP / 8; ++h) {
            float o[8];
            ld8(k < DA ? sa : sb, vk, LP, h, o);
            acc8<LP, F2>(ky, h, wk, o);
        }
    }
}

// One chunk: every pixel of it (see the comment above PixArgs).
// Returns false (for the whole block) when the chunk's tile copy did not
// complete within both bounded waits: DCRF_E_TIMEOUT is then flagged, the
// block touches neither the tile nor y, s and the splat, and the launch's
// outputs are invalid.
template <int LP, typename TB, bool POTTS, int MODE>
__device__ __forceinline__ bool pixel_chunk(const PixArgs &A, const FwLats &F, const Chunk &ch, float *sy,
                                            const float *sl, float (&part)[NS], unsigned long long *tbar) {
    const int L = (MODE & kL21) ? 21 : A.L;
    const bool start = A.alpha == nullptr;
    const float al = start ? 0.f : (float)A.alpha[ch.image];
#pragma unroll
    for (int q = 0; q < NS; ++q) part[q] = 0.f;
    const int t = threadIdx.x;
    const bool valid = t < ch.count;
    const int64_t a = ch.begin + (valid ? t : 0);
    const float *yrow = sy + t * A.Ls;
    const float *lrow = sl + t * A.Ls;
    int sb = 0;
    float ky[LP];
#pragma unroll
    for (int i = 0; i < LP; ++i) ky[i] = 0.f;
    int sold = -1;
    if (valid) {
        if (!start) sold = A.s[a];
        // K~ y' gathered from the lattice, eight labels at a time
        constexpr bool F2 = (MODE & kF2) != 0;
        const bool fixed = (MODE & kFix) && F.nk == 2 && F.l[0].d1 == 6 && F.l[1].d1 == 3;
        if (fixed) gather_pair<LP, TB, 6, 3, F2>(F.l[0], F.l[1], a, ky);
#pragma unroll
        for (int mm = 0; mm < DCRF_MAX_KERNELS; ++mm) {
            if (fixed || mm >= F.nk) break;
            const FwLat &lt = F.l[mm];
            const TB *src = slice_src<TB>(lt);
            for (int k = 0; k < lt.d1; ++k) {
                const int v = __ldg(lt.pvid + a * lt.d1 + k);
                if (v < 0) continue;
                const float w = __ldg(lt.pbary + a * lt.d1 + k) * lt.ws0;
#pragma unroll
                for (int h = 0; h < LP / 8; ++h) {
                    float o[8];
                    ld8(src, v, LP, h, o);
                    acc8<LP, F2>(ky, h, w, o);
                }
            }
        }
    }
    bool tile_ok = true;
    if constexpr ((MODE & kEarly) != 0) {
        // the tile copies were left in flight during the gather
        if (tbar) {
            if (!mbar_wait(tbar)) {
                // report, then wait (bounded, longer) for the copies still in flight
                dcrf_flag(A.status, DCRF_E_TIMEOUT);
                tile_ok = mbar_wait(tbar, kWaitPollsLast);
            }
        } else {
            cp_wait<0>();
        }
        tile_ok = __syncthreads_and(tile_ok) != 0;
    }
    if (!tile_ok) {
#pragma unroll
        for (int q = 0; q < NS; ++q) part[q] = 0.f;
        return false;
    }
    if (valid) {
      if constexpr (POTTS && (MODE & kLean) != 0) {
        // Potts, one pass for y' and the totals, then the argmin tracking only
        // (g, s', X(s')); lin(s'), y'(s') are read back and P(s') recomputed
        // with the same operations, so every result is the same as below
        float *yw = sy + t * A.Ls;
        const float ca = A.c[a];
        float tot = 0.f, sy_ = 0.f;
#pragma unroll
        for (int i = 0; i < LP; ++i) {
            if (i < L) {
                float y = yw[i];
                if (!start) {
                    y = y + al * ((i == sold ? 1.f : 0.f) - y);
                    yw[i] = y;
                }
                ky[i] -= A.sumw * y;          // X = K~ y' - sum_w y'
                tot += ky[i];
                sy_ += y;
            }
        }
        const float dpot = (float)(L - 1) * ca;
        float best = INFINITY, kys = 0.f;
        float s0 = 0.f, s1 = 0.f, s6 = 0.f;
#pragma unroll
        for (int i = 0; i < LP; ++i) {
            if (i < L) {
                const float y = yrow[i];
                const float P = (tot - ky[i]) + dpot * y;
                const float li = lrow[i];
                const float g = li + 2.f * P;
                if (g < best) { best = g; sb = i; kys = ky[i]; }
                s0 += li * y;
                s1 += y * P;
                s6 += dpot * y * y;
            }
        }
        if (!(best < INFINITY)) dcrf_flag(A.status, DCRF_E_NONFINITE);
        const float y_s = yrow[sb], lin_s = lrow[sb];
        const float P_s = (tot - kys) + dpot * y_s;
        part[0] = s0;
        part[1] = s1;
        part[2] = lin_s;
        part[3] = P_s;
        part[4] = -A.sumw * (sy_ - y_s) + y_s * dpot;
        part[5] = dpot;
        part[6] = s6;
        if (A.phi) {
            float sp = 0.f;
#pragma unroll
            for (int i = 0; i < LP; ++i)
                if (i < L) sp += A.phi[a * L + i] * yrow[i];
            part[7] = sp;
        }
      } else {
        // y' = y + alpha (e_sold - y), written over the thread's shared-memory
        // row once (it is stored back to Y after the block)
        if (!start) {
            float *yw = sy + t * A.Ls;
#pragma unroll
            for (int i = 0; i < LP; ++i)
                if (i < L) {
                    const float v = yw[i];
                    yw[i] = v + al * ((i == sold ? 1.f : 0.f) - v);
                }
        }
        auto yp = [&](int i) { return yrow[i]; };
        const float ca = A.c[a];
        float tot = 0.f, sy_ = 0.f;
#pragma unroll
        for (int i = 0; i < LP; ++i) {
            if (i < L) {
                const float y = yp(i);
                ky[i] -= A.sumw * y;          // X = K~ y' - sum_w y'
                tot += ky[i];
                sy_ += y;
            }
        }
        if (!POTTS) {
            float X[LP];
#pragma unroll
            for (int i = 0; i < LP; ++i) X[i] = ky[i];
#pragma unroll
            for (int i = 0; i < LP; ++i) {
                if (i < L) {
                    float acc = 0.f;
#pragma unroll 8
                    for (int j = 0; j < LP; ++j)
                        if (j < L) acc += A.mu[i * L + j] * X[j];
                    ky[i] = acc;              // mu X
                }
            }
        }
        const float dpot = (float)(L - 1) * ca;
        float best = INFINITY;
        float s0 = 0.f, s1 = 0.f, s6 = 0.f;
        float lin_s = 0.f, P_s = 0.f, y_s = 0.f;
#pragma unroll
        for (int i = 0; i < LP; ++i) {
            if (i < L) {
                const float y = yp(i);
                const float di = POTTS ? dpot : A.musum[i] * ca;
                const float P = (POTTS ? tot - ky[i] : ky[i]) + di * y;    // (Psi + D) y'
                const float li = lrow[i];
                const float g = li + 2.f * P;
                if (g < best) { best = g; sb = i; lin_s = li; P_s = P; y_s = y; }
                s0 += li * y;
                s1 += y * P;
                s6 += di * y * y;
            }
        }
        if (!(best < INFINITY)) dcrf_flag(A.status, DCRF_E_NONFINITE);
        float ymu, mu_ss;   // <y', mu e_s'>, mu(s', s')
        if (POTTS) {
            ymu = sy_ - y_s;
            mu_ss = 0.f;
        } else {
            ymu = 0.f;
#pragma unroll
            for (int i = 0; i < LP; ++i)
                if (i < L) ymu += yp(i) * A.mu[i * L + sb];
            mu_ss = A.mu[sb * L + sb];
        }
        const float ds = POTTS ? dpot : A.musum[sb] * ca;
        part[0] = s0;
        part[1] = s1;
        part[2] = lin_s;
        part[3] = P_s;
        part[4] = -A.sumw * ymu + y_s * ds;
        part[5] = -A.sumw * mu_ss + ds;
        part[6] = s6;
        if (A.phi) {
            float sp = 0.f;
#pragma unroll
            for (int i = 0; i < LP; ++i)
                if (i < L) sp += A.phi[a * L + i] * yp(i);
            part[7] = sp;
        }
      }
        A.s[a] = (uint8_t)sb;
        // splat of the one-hot s' into Sq (integer reductions in L2).  A delta
        // update (+b at s', -b at s) does not pay: along the Frank-Wolfe path
        // almost every pixel's argmin moves at every iteration.
#pragma unroll
        for (int mm = 0; mm < DCRF_MAX_KERNELS; ++mm) {
            if (mm >= F.nk) break;
            const FwLat &lt = F.l[mm];
            const float q = __ldg(lt.qs);
            for (int k = 0; k < lt.d1; ++k) {
                const int v = __ldg(lt.pvid + a * lt.d1 + k);
                if (v >= 0) atomicAdd(lt.St + (int64_t)v * LP + sb, __float2uint_rn(q * __ldg(lt.pbary + a * lt.d1 + k)));
            }
        }
    }
    return true;
}

// Label-split layout of the pixel pass (Lp = 24, Potts): three lanes per
// pixel, lane q of a pixel owns labels 8q .. 8q+7, so one warp instruction
// gathers ten whole 48-byte (FP16) corner rows instead of one 16-byte piece
// of 32 different rows.  Lanes 30 and 31 of each warp are idle; a warp holds
// ten pixels.  Same sums and splat as pixel_chunk: the per-pixel scalars
// (total over labels, argmin) are combined over the three lanes in a fixed
// order, so the lanes of a pixel agree bit for bit.
constexpr int kL3Warps = 8;                 // warps per block
constexpr int kL3Pixels = 10 * kL3Warps;    // pixels per block

template <typename TB>
__device__ __forceinline__ void pixel3(const PixArgs &A, const FwLats &F, const Chunk &ch, float *sy,
                                       const float *sl, float (&part)[NS]) {
    constexpr int LP = 24;
    const int L = A.L;
    const bool start = A.alpha == nullptr;
    const float al = start ? 0.f : (float)A.alpha[ch.image];
#pragma unroll
    for (int q = 0; q < NS; ++q) part[q] = 0.f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / 3, q = lane - 3 * (lane / 3);
    const int px = 10 * warp + g;                        // pixel within the chunk
    const bool valid = lane < 30 && px < ch.count;
    const int64_t a = ch.begin + (valid ? px : 0);
    const int base = 3 * (lane < 30 ? g : 9);            // first lane of this pixel's group
    float *yw = sy + (valid ? px : 0) * A.Ls;
    const float *lrow = sl + (valid ? px : 0) * A.Ls;
    float ky[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) ky[j] = 0.f;
    int sold = -1;
    if (valid) {
        if (!start) sold = A.s[a];
        const bool fixed = F.nk == 2 && F.l[0].d1 == 6 && F.l[1].d1 == 3;
        if (fixed) {
            int v[9];
            float w[9];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                v[k] = __ldg(F.l[0].pvid + a * 6 + k);
                w[k] = __ldg(F.l[0].pbary + a * 6 + k) * F.l[0].ws0;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                v[6 + k] = __ldg(F.l[1].pvid + a * 3 + k);
                w[6 + k] = __ldg(F.l[1].pbary + a * 3 + k) * F.l[1].ws0;
            }
            const TB *s0p = slice_src<TB>(F.l[0]), *s1p = slice_src<TB>(F.l[1]);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int vk = v[k] < 0 ? 0 : v[k];
                const float wk = v[k] < 0 ? 0.f : w[k];
                float o[8];
                ld8(k < 6 ? s0p : s1p, vk, LP, q, o);
#pragma unroll
                for (int j = 0; j < 8; ++j) ky[j] += wk * o[j];
            }
        } else {
#pragma unroll
            for (int mm = 0; mm < DCRF_MAX_KERNELS; ++mm) {
                if (mm >= F.nk) break;
                const FwLat &lt = F.l[mm];
                const TB *src = slice_src<TB>(lt);
                for (int k = 0; k < lt.d1; ++k) {
                    const int v = __ldg(lt.pvid + a * lt.d1 + k);
                    if (v < 0) continue;
                    const float w = __ldg(lt.pbary + a * lt.d1 + k) * lt.ws0;
                    float o[8];
                    ld8(src, v, LP, q, o);
#pragma unroll
                    for (int j = 0; j < 8; ++j) ky[j] += w * o[j];
                }
            }
        }
        // y' over this lane's labels, written back to the shared row
        if (!start) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int i = 8 * q + j;
                if (i < L) {
                    const float yv = yw[i];
                    yw[i] = yv + al * ((i == sold ? 1.f : 0.f) - yv);
                }
            }
        }
    }
    // totals over the pixel's labels: X = K~ y' - sum_w y', sum X, sum y'
    float ptot = 0.f, psy = 0.f;
    if (valid) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = 8 * q + j;
            if (i < L) {
                const float y = yw[i];
                ky[j] -= A.sumw * y;
                ptot += ky[j];
                psy += y;
            }
        }
    }
    const float t0 = __shfl_sync(0xffffffffu, ptot, base), t1 = __shfl_sync(0xffffffffu, ptot, base + 1),
                t2 = __shfl_sync(0xffffffffu, ptot, base + 2);
    const float y0s = __shfl_sync(0xffffffffu, psy, base), y1s = __shfl_sync(0xffffffffu, psy, base + 1),
                y2s = __shfl_sync(0xffffffffu, psy, base + 2);
    const float tot = (t0 + t1) + t2, sy_ = (y0s + y1s) + y2s;
    const float ca = valid ? A.c[a] : 0.f;
    const float dpot = (float)(L - 1) * ca;
    float best = INFINITY;
    int sb = 0;
    float lin_s = 0.f, P_s = 0.f, y_s = 0.f;
    float s0 = 0.f, s1 = 0.f, s6 = 0.f, sp = 0.f;
    if (valid) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = 8 * q + j;
            if (i < L) {
                const float y = yw[i];
                const float P = (tot - ky[j]) + dpot * y;      // (Psi + D) y'
                const float li = lrow[i];
                const float gi = li + 2.f * P;
                if (gi < best) { best = gi; sb = i; lin_s = li; P_s = P; y_s = y; }
                s0 += li * y;
                s1 += y * P;
                s6 += dpot * y * y;
                if (A.phi) sp += A.phi[a * L + i] * y;
            }
        }
    }
    // argmin over the three lanes (lowest label on ties: lane order is label order)
    const float b0 = __shfl_sync(0xffffffffu, best, base), b1 = __shfl_sync(0xffffffffu, best, base + 1),
                b2 = __shfl_sync(0xffffffffu, best, base + 2);
    int win = 0;
    float bw = b0;
    if (b1 < bw) { bw = b1; win = 1; }
    if (b2 < bw) { bw = b2; win = 2; }
    const int sbw = __shfl_sync(0xffffffffu, sb, base + win);
    if (valid) {
        if (!(bw < INFINITY) && q == 0) dcrf_flag(A.status, DCRF_E_NONFINITE);
        part[0] = s0;
        part[1] = s1;
        part[6] = s6;
        part[7] = sp;
        if (q == win) {
            part[2] = lin_s;
            part[3] = P_s;
            part[4] = -A.sumw * (sy_ - y_s) + y_s * dpot;   // Potts: <y', mu e_s'> = sum y' - y'(s')
            part[5] = dpot;                                  // mu(s', s') = 0
        }
        if (q == 0) A.s[a] = (uint8_t)sbw;
        // splat of the one-hot s': lane q takes corners k = q, q + 3, ...
#pragma unroll
        for (int mm = 0; mm < DCRF_MAX_KERNELS; ++mm) {
            if (mm >= F.nk) break;
            const FwLat &lt = F.l[mm];
            const float qk = __ldg(lt.qs);
            for (int k = q; k < lt.d1; k += 3) {
                const int v = __ldg(lt.pvid + a * lt.d1 + k);
                if (v >= 0)
                    atomicAdd(lt.St + (int64_t)v * LP + sbw, __float2uint_rn(qk * __ldg(lt.pbary + a * lt.d1 + k)));
            }
        }
    }
}

template <typename TB>
__global__ void __launch_bounds__(32 * kL3Warps) k_fw_pixel3(PixArgs A, FwLats F) {
    extern __shared__ __align__(16) float smem[];
    float *sy = smem;
    float *sl = smem + kL3Pixels * A.Ls;
    const Chunk ch = A.chunks[blockIdx.x];
    tile_load_async(A, ch, sy, sl);
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    float part[NS];
    pixel3<TB>(A, F, ch, sy, sl, part);
    __syncthreads();
    if (A.alpha != nullptr) tile_store(A, ch, sy);
    warp_sums<NS>(part, A.cpart + (int64_t)blockIdx.x * kL3Warps * NS);
}

// One block per chunk: the chunk's y and lin rows are copied to shared memory
// (cp.async), every pixel is processed, y' is written back coalesced.
template <int LP, typename TB, bool POTTS, int PB, int MB, int MODE>
__global__ void __launch_bounds__(PB, MB) k_fw_pixel(PixArgs A, FwLats F) {
    extern __shared__ __align__(16) float smem[];
    float *sy = smem;
    float *sl = smem + PB * A.Ls;
    const Chunk ch = A.chunks[blockIdx.x];
    __shared__ __align__(8) unsigned long long tbar_s;
    unsigned long long *tbar = nullptr;
    if constexpr ((MODE & kBulk) != 0) {
        static_assert((MODE & kEarly) != 0, "bulk tiles wait in the early-gather path");
        if (tile_bulk_ok(A, ch)) tbar = &tbar_s;     // uniform over the block
    }
    if (tbar) {
        if (threadIdx.x == 0) mbar_init(tbar);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int64_t base = ch.begin * (int64_t)A.L;
            const unsigned bytes = (unsigned)(ch.count * A.L) * 4u;
            mbar_expect_tx(tbar, 2u * bytes);
            bulk_g2s(sy, A.Y + base, bytes, tbar);
            bulk_g2s(sl, A.lin + base, bytes, tbar);
        }
    } else {
        tile_load_async(A, ch, sy, sl);
        cp_commit();
        if constexpr ((MODE & kEarly) == 0) {
            cp_wait<0>();
            __syncthreads();
        }
    }
    float part[NS];
    const bool tile_ok = pixel_chunk<LP, TB, POTTS, MODE>(A, F, ch, sy, sl, part, tbar);
    if (tbar) fence_proxy_async_smem();   // y' rows written here are read by the bulk store
    __syncthreads();
    if (A.alpha != nullptr && tile_ok) {
        if (tbar) {
            if (threadIdx.x == 0)
                bulk_s2g(A.Y + ch.begin * (int64_t)A.L, sy, (unsigned)(ch.count * A.L) * 4u);
        } else {
            tile_store(A, ch, sy);
        }
    }
    warp_sums<NS>(part, A.cpart + (int64_t)blockIdx.x * (PB / 32) * NS);
}

}  // namespace
