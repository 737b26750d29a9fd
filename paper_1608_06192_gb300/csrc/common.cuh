// Shared definitions of the dense-CRF CUDA path (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <vector>

#include "dcrf.h"

#define DCRF_MAX_D 8
#define DCRF_MAX_L 64
#define DCRF_MAX_KERNELS 4

#define DCRF_TRY(expr)                                                     \
    do {                                                                   \
        cudaError_t e__ = (expr);                                          \
        if (e__ != cudaSuccess) {                                          \
            return e__ == cudaErrorMemoryAllocation ? DCRF_E_NOMEM : DCRF_E_CUDA; \
        }                                                                  \
    } while (0)

#define DCRF_LAUNCHED()                                                    \
    do {                                                                   \
        cudaError_t e__ = cudaGetLastError();                              \
        if (e__ != cudaSuccess) return DCRF_E_CUDA;                        \
    } while (0)

#define DCRF_CHECK_STATUS(expr)                                            \
    do {                                                                   \
        dcrf_status st__ = (expr);                                         \
        if (st__ != DCRF_OK) return st__;                                  \
    } while (0)

// Empty hash slot.  Packed keys never reach it: every coordinate field is
// kept below its all-ones value.
#define DCRF_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull

struct dcrf_lattice_s {
    int d = 0;
    int64_t n = 0;
    int64_t m = 0;
    int batch = 0;
    double s0 = 1.0;                 // output scale of the slice
    double s1max = 0.0;              // max over vertices of (S 1)_v, the summed barycentric weights
    std::vector<int64_t> point_off;  // host [batch+1]
    std::vector<int64_t> vert_off;   // host [batch+1]
    int64_t *point_off_d = nullptr;  // device [batch+1]
    int64_t *vert_off_d = nullptr;   // device [batch+1]
    int32_t *pvid = nullptr;         // [n][d+1] vertex of each simplex corner
    float *pbary = nullptr;          // [n][d+1] barycentric weight of that corner
    int32_t *keys = nullptr;         // [m][d]
    int32_t *nbr = nullptr;          // [m][d+1][2]
    int32_t *vimg = nullptr;         // [m] image of each vertex
    float *ones = nullptr;           // [n] (K~_lattice 1)_a, s0 included
    int *status = nullptr;           // device status word (first error wins)
    int device = -1;                 // the device whose memory pool holds the arrays
};

// Records the first device-side error.
__device__ __forceinline__ void dcrf_flag(int *status, int code) {
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint64_t dcrf_hash64(uint64_t k) {
    // splitmix64 finaliser
    k ^= k >> 30;
    k *= 0xbf58476d1ce4e5b9ull;
    k ^= k >> 27;
    k *= 0x94d049bb133111ebull;
    k ^= k >> 31;
    return k;
}

__host__ __device__ __forceinline__ int dcrf_key_bits(int d) {
    int b = 64 / d;
    return b > 32 ? 32 : b;
}

// Work chunk: a contiguous range of rows inside one image.
struct Chunk {
    int64_t begin;
    int32_t count;
    int32_t image;
};

// Splits each image's row range into chunks of at most `size` rows.
std::vector<Chunk> make_chunks(const std::vector<int64_t> &off, int size);

// Host helpers (lattice.cu).
dcrf_status dcrf_check_lattices(const dcrf_lattice *lats, int n_k);
int dcrf_round4(int L);

// The library's caching pool for the stream's device (pool.cu), or NULL for
// the default pool (while the stream is captured, or when DCRF_POOL=default).
cudaMemPool_t dcrf_scratch_pool(cudaStream_t s);

template <typename T>
dcrf_status dcrf_alloc(T **p, size_t count, cudaStream_t s) {
    *p = nullptr;
    if (count == 0) return DCRF_OK;
    cudaMemPool_t pool = dcrf_scratch_pool(s);
    cudaError_t e = pool ? cudaMallocFromPoolAsync((void **)p, count * sizeof(T), pool, s)
                         : cudaMallocAsync((void **)p, count * sizeof(T), s);
    if (e != cudaSuccess) { *p = nullptr; return DCRF_E_NOMEM; }
    return DCRF_OK;
}

// Stream-ordered scratch owned by one call; freed on the same stream.
struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <typename T>
    dcrf_status get(T **p, size_t count) {
        dcrf_status st = dcrf_alloc(p, count, s);
        if (st == DCRF_OK && *p) ptrs.push_back((void *)*p);
        return st;
    }
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
    }
};

dcrf_status dcrf_fill(float *p, float v, int64_t n, cudaStream_t s);

// Per-kernel event timing (profile.cu); ids index the name table there.
enum ProfId {
    P_EMBED = 0, P_FINALIZE, P_NEIGHBOURS, P_SPLAT_DENSE, P_BLUR, P_SLICE,
    P_FW_PIXEL, P_FW_LATDOT, P_FW_ALPHA, P_FW_LATUPD, P_FW_LIN,
    P_LP_SORT, P_LP_RUNS, P_LP_SPLAT, P_LP_NEIGHBOURS, P_LP_BLUR, P_LP_SLICE, P_LP_COMBINE,
    P_LP_PROJECT, P_LP_LOCAL, P_FW_BLUR, P_DCNEG_PIXEL
};
struct ProfScope {
    ProfScope(int id, cudaStream_t s);
    ~ProfScope();
    int id_;
    cudaStream_t s_;
    void *a_;
};
bool dcrf_profiling();

// Filter pipeline pieces shared by the solvers (lattice.cu).
// Splat Y [n][L] (float32 rows) into V [m][Lp] float32 (V must be zeroed).
dcrf_status dcrf_splat_dense(const dcrf_lattice lat, const float *Y, int L, float *V, int Lp,
                             cudaStream_t s);
// The d+1 blur passes (axis order 0..d, or d..0 when reverse).  src is
// float32 [m][Lp]; the result lands in dst (float or half per storage); tmp is
// scratch of the same type as dst.  src is left intact.
dcrf_status dcrf_blur(const dcrf_lattice lat, const float *src, void *dst, void *tmp, int Lp,
                      int storage, bool reverse, cudaStream_t s);
// out [n][L] = s0 * slice of lattice values V [m][Lp] (float32, or float16
// when storage is DCRF_STORAGE_F16).
dcrf_status dcrf_slice(const dcrf_lattice lat, const void *V, int Lp, int L, int storage, float *out,
                       cudaStream_t s);
dcrf_status dcrf_slice_f32(const dcrf_lattice lat, const float *V, int Lp, int L, float *out, cudaStream_t s);
// Stable radix sort of (key, value) pairs inside host-given segments
// [seg_begin[s], seg_begin[s+1]) by the low `bits` key bits (segsort.cu);
// the result lands in kout/vout, ktmp/vtmp are scratch, kin/vin are read only.
dcrf_status dcrf_segsort(const uint32_t *kin, const int32_t *vin, uint32_t *ktmp, int32_t *vtmp, uint32_t *kout,
                         int32_t *vout, const int64_t *seg_begin, int nseg, int bits, cudaStream_t s);
// idx / cols for 0 <= idx < count: the 32-bit division when count fits 32
// bits (a branch that is uniform over the launch), else the 64-bit one, whose
// long instruction sequence dominated the element-wise kernels that index
// [rows][cols] arrays by a flat index.
__device__ __forceinline__ int64_t dcrf_div(int64_t idx, int cols, int64_t count) {
    return count <= 0xffffffffll ? (int64_t)((uint32_t)idx / (uint32_t)cols) : idx / cols;
}
// Prefix sums of integer arrays (scan.cu): out[i] = sum of in[0 .. i)
// (exclusive) or in[0 .. i] (inclusive); out may not alias in.
dcrf_status dcrf_scan(const int32_t *in, int32_t *out, int64_t n, bool inclusive, cudaStream_t s);
dcrf_status dcrf_scan(const uint32_t *in, int64_t *out, int64_t n, bool inclusive, cudaStream_t s);
// Looks up, once per device, the device address of dcrf_filter_static's
// array for the device of stream s (noalloc.cu).
dcrf_status dcrf_static_scratch(cudaStream_t s, unsigned char **out);
