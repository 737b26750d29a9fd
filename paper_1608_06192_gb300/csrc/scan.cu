// Device-wide prefix sums (exclusive or inclusive) of integer arrays.
//
// Used where the lattice build counts the vertices of each image and numbers
// them, and where the LP divide and conquer numbers the runs of tagged
// vertices and the incidences of every vertex.  Reduce-then-scan over tiles of
// kTile elements: the tile sums, their exclusive scan (recursively, one block
// once there are at most kTile of them), then every tile scanned again with
// its offset added.  Integer sums are exact, so the result does not depend on
// the tiling.
#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;   // 4096
constexpr int kWarpSpan = kTile / kWarps;  // 512 contiguous elements per warp

// Warp w of a block owns elements [w kWarpSpan, (w+1) kWarpSpan) of the tile
// and reads them in kItems rounds of 32 consecutive elements (coalesced):
// element (round r, lane l) is w kWarpSpan + 32 r + l, so (warp, round, lane)
// order is the input order.
template <typename Tin, typename Tout>
__device__ __forceinline__ void load_tile(const Tin *__restrict__ in, int64_t n, int64_t tile, Tout (&v)[kItems]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = tile * kTile + (int64_t)warp * kWarpSpan + lane;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t i = base + 32 * r;
        v[r] = i < n ? (Tout)in[i] : (Tout)0;
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads) k_tile_sums(const Tin *__restrict__ in, int64_t n, Tout *__restrict__ sums) {
    __shared__ Tout warp_tot[kWarps];
    Tout v[kItems];
    load_tile<Tin, Tout>(in, n, blockIdx.x, v);
    Tout acc = 0;
#pragma unroll
    for (int r = 0; r < kItems; ++r) acc += v[r];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        Tout t = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += warp_tot[w];
        sums[blockIdx.x] = t;
    }
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const Tin *__restrict__ in, int64_t n,
                                                        const Tout *__restrict__ offs, bool inclusive,
                                                        Tout *__restrict__ out) {
    __shared__ Tout warp_tot[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Tout v[kItems];
    load_tile<Tin, Tout>(in, n, blockIdx.x, v);
    Tout acc = 0;
#pragma unroll
    for (int r = 0; r < kItems; ++r) acc += v[r];
    acc = warp_sum(acc);
    if (lane == 0) warp_tot[warp] = acc;
    __syncthreads();
    Tout carry = offs ? offs[blockIdx.x] : (Tout)0;   // sum of everything before this warp's span
    for (int w = 0; w < warp; ++w) carry += warp_tot[w];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)warp * kWarpSpan + lane;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        Tout inc = v[r];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const Tout x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += x;
        }
        const int64_t i = base + 32 * r;
        if (i < n) out[i] = carry + (inclusive ? inc : inc - v[r]);
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
}

template <typename Tin, typename Tout>
dcrf_status scan_impl(const Tin *in, Tout *out, int64_t n, bool inclusive, cudaStream_t s) {
    if (n <= 0) return DCRF_OK;
    const int64_t tiles = (n + kTile - 1) / kTile;
    if (tiles > (1ll << 31) - 1) return DCRF_E_INVAL;
    Tout *offs = nullptr;
    Scratch sc(s);
    if (tiles > 1) {
        Tout *sums;
        DCRF_CHECK_STATUS(sc.get(&sums, (size_t)tiles));
        DCRF_CHECK_STATUS(sc.get(&offs, (size_t)tiles));
        k_tile_sums<Tin, Tout><<<(unsigned)tiles, kThreads, 0, s>>>(in, n, sums);
        DCRF_LAUNCHED();
        DCRF_CHECK_STATUS((scan_impl<Tout, Tout>(sums, offs, tiles, false, s)));
    }
    k_tile_scan<Tin, Tout><<<(unsigned)tiles, kThreads, 0, s>>>(in, n, offs, inclusive, out);
    DCRF_LAUNCHED();
    return DCRF_OK;
}

}  // namespace

dcrf_status dcrf_scan(const int32_t *in, int32_t *out, int64_t n, bool inclusive, cudaStream_t s) {
    return scan_impl<int32_t, int32_t>(in, out, n, inclusive, s);
}
dcrf_status dcrf_scan(const uint32_t *in, int64_t *out, int64_t n, bool inclusive, cudaStream_t s) {
    return scan_impl<uint32_t, int64_t>(in, out, n, inclusive, s);
}
