// Stable segmented radix sort of (uint32 key, int32 value) pairs.
//
// The LP subgradient (Section 6, Eq. 19, Algorithm 3) orders every label
// column of every image by descending y_a(i), ties by ascending pixel index,
// and groups the lattice incidences of each (label, image) by vertex in rank
// order (Appendix E).  Both are stable sorts inside segments that the host
// knows: this file sorts them with least-significant-digit radix passes of
// 8 bits.  Each segment is cut into tiles of kTile elements that never cross
// a segment boundary; a pass is
//   1. k_ss_hist    one block per tile: digit histogram of the tile;
//   2. k_ss_offsets one block per segment: for every (tile, digit) the output
//                   position of the tile's first element with that digit
//                   (digits in order, tiles in order: the pass is stable);
//   3. k_ss_scatter one block per tile: the stable rank of each element among
//                   the tile's elements with its digit (warp multisplit with
//                   __match_any_sync, warps in order), written to its place.
// Keys are compared as unsigned integers; callers map their values to keys
// whose ascending order is the wanted one.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                      // per thread
constexpr int kTile = kThreads * kItems;        // 4096 elements
constexpr int kWarpSpan = kTile / kWarps;       // contiguous elements of one warp (512)
constexpr int kRadix = 256;

struct Tile {
    int64_t begin;   // first element
    int32_t count;   // elements (<= kTile)
    int32_t seg;     // segment
};

__global__ void __launch_bounds__(kThreads) k_ss_hist(const uint32_t *__restrict__ keys, const Tile *__restrict__ tiles,
                                                      int shift, uint32_t mask, uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[kRadix];
    const Tile t = tiles[blockIdx.x];
    h[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < t.count; i += kThreads) atomicAdd(&h[(keys[t.begin + i] >> shift) & mask], 1u);
    __syncthreads();
    hist[(int64_t)blockIdx.x * kRadix + threadIdx.x] = h[threadIdx.x];
}

// Segment s owns tiles [tile0[s], tile0[s+1]) and elements from seg_begin[s];
// off[t][d] = seg_begin + (elements of the segment with a smaller digit) +
// (elements with digit d in the segment's earlier tiles).
__global__ void __launch_bounds__(kThreads) k_ss_offsets(const uint32_t *__restrict__ hist,
                                                         const int32_t *__restrict__ tile0,
                                                         const int64_t *__restrict__ seg_begin,
                                                         int64_t *__restrict__ off) {
    __shared__ uint32_t warp_tot[kWarps];
    const int s = blockIdx.x, d = threadIdx.x;
    const int t0 = tile0[s], t1 = tile0[s + 1];
    uint32_t total = 0;
    for (int t = t0; t < t1; ++t) total += hist[(int64_t)t * kRadix + d];
    // exclusive scan of the digit totals over the block (digit order)
    const int lane = d & 31, warp = d >> 5;
    uint32_t inc = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    int64_t run = seg_begin[s] + before + inc - total;
    for (int t = t0; t < t1; ++t) {
        off[(int64_t)t * kRadix + d] = run;
        run += hist[(int64_t)t * kRadix + d];
    }
}

__global__ void __launch_bounds__(kThreads) k_ss_scatter(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                                                         const Tile *__restrict__ tiles, const int64_t *__restrict__ off,
                                                         int shift, uint32_t mask, uint32_t *__restrict__ kout,
                                                         int32_t *__restrict__ vout) {
    __shared__ uint32_t cnt[kWarps][kRadix];
    const Tile t = tiles[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[kItems];
    int32_t val[kItems];
    uint32_t rank[kItems];
    // warp `warp` takes elements [warp * kWarpSpan, (warp + 1) * kWarpSpan) of
    // the tile, 32 at a time: (round, lane) order is the input order
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int i = warp * kWarpSpan + r * 32 + lane;
        const bool ok = i < t.count;
        key[r] = ok ? kin[t.begin + i] : 0u;
        val[r] = ok ? vin[t.begin + i] : 0;
        const uint32_t dg = ok ? (key[r] >> shift) & mask : kRadix;   // kRadix: no element
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t base = ok ? cnt[warp][dg] : 0u;
        rank[r] = base + __popc(peers & lt);
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) cnt[warp][dg] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // counts of the earlier warps, per digit (warps in element order)
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const int64_t *to = off + (int64_t)blockIdx.x * kRadix;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int i = warp * kWarpSpan + r * 32 + lane;
        if (i < t.count) {
            const uint32_t dg = (key[r] >> shift) & mask;
            const int64_t p = to[dg] + cnt[warp][dg] + rank[r];
            kout[p] = key[r];
            vout[p] = val[r];
        }
    }
}

}  // namespace

// Sorts the pairs of every segment [seg_begin[s], seg_begin[s+1]) (host
// array, nseg + 1 entries, non-decreasing) by key, stably, using the low
// `bits` bits of the keys.  kin/vin are read only; the result lands in
// kout/vout; ktmp/vtmp are scratch of the same size; the tile tables are
// taken from the stream-ordered pool and given back before the return.
// Elements outside every segment are neither read nor written.
dcrf_status dcrf_segsort(const uint32_t *kin, const int32_t *vin, uint32_t *ktmp, int32_t *vtmp, uint32_t *kout,
                         int32_t *vout, const int64_t *seg_begin, int nseg, int bits, cudaStream_t s) {
    if (nseg < 1 || bits < 1 || bits > 32) return DCRF_E_INVAL;
    std::vector<Tile> tiles;
    std::vector<int32_t> tile0(nseg + 1, 0);
    for (int g = 0; g < nseg; ++g) {
        tile0[g] = (int32_t)tiles.size();
        for (int64_t b = seg_begin[g]; b < seg_begin[g + 1]; b += kTile)
            tiles.push_back(Tile{b, (int32_t)std::min<int64_t>(kTile, seg_begin[g + 1] - b), g});
    }
    tile0[nseg] = (int32_t)tiles.size();
    const int64_t nt = (int64_t)tiles.size();
    if (nt == 0) return DCRF_OK;
    Scratch sc(s);   // released (stream-ordered) when the sort's kernels are done
    if (nt >= (1ll << 31) / kRadix) return DCRF_E_INVAL;
    Tile *tiles_d;
    int32_t *tile0_d;
    int64_t *segb_d, *off;
    uint32_t *hist;
    DCRF_CHECK_STATUS(sc.get(&tiles_d, (size_t)nt));
    DCRF_CHECK_STATUS(sc.get(&tile0_d, (size_t)nseg + 1));
    DCRF_CHECK_STATUS(sc.get(&segb_d, (size_t)nseg + 1));
    DCRF_CHECK_STATUS(sc.get(&hist, (size_t)nt * kRadix));
    DCRF_CHECK_STATUS(sc.get(&off, (size_t)nt * kRadix));
    DCRF_TRY(cudaMemcpyAsync(tiles_d, tiles.data(), nt * sizeof(Tile), cudaMemcpyHostToDevice, s));
    DCRF_TRY(cudaMemcpyAsync(tile0_d, tile0.data(), (nseg + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DCRF_TRY(cudaMemcpyAsync(segb_d, seg_begin, (nseg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const int passes = (bits + 7) / 8;
    const uint32_t *ks = kin;
    const int32_t *vs = vin;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        const int w = std::min(8, bits - shift);
        const uint32_t mask = (1u << w) - 1u;
        // the last pass lands in kout
        uint32_t *kd = ((passes - 1 - p) % 2 == 0) ? kout : ktmp;
        int32_t *vd = ((passes - 1 - p) % 2 == 0) ? vout : vtmp;
        k_ss_hist<<<(unsigned)nt, kThreads, 0, s>>>(ks, tiles_d, shift, mask, hist);
        DCRF_LAUNCHED();
        k_ss_offsets<<<nseg, kThreads, 0, s>>>(hist, tile0_d, segb_d, off);
        DCRF_LAUNCHED();
        k_ss_scatter<<<(unsigned)nt, kThreads, 0, s>>>(ks, vs, tiles_d, off, shift, mask, kd, vd);
        DCRF_LAUNCHED();
        ks = kd;
        vs = vd;
    }
    return DCRF_OK;
}
