// dcrf_filter_static: the lattice filter without any device allocation.
//
// dcrf_filter takes its lattice-value scratch (a splat buffer and two blur
// buffers) from the stream-ordered allocator on every call.  Some callers
// cannot allocate device memory at that point: code that runs while a stream
// is being captured into a CUDA graph under a mode that forbids allocation,
// real-time loops with a fixed memory budget, or hosts whose allocator is not
// reachable from the calling thread.  This variant computes the same K~ Y but
// places its scratch in one file-scope device array of fixed size, so a call
// launches kernels and a memset and nothing else.
//
// The array (DCRF_STATIC_SCRATCH_BYTES) is reserved on every GPU that loads
// the library, for the life of the process.  Every call uses the same array
// and finds the previous call's contents there; the splat buffer is cleared
// at the start of each call.  Two calls whose work overlaps on the GPU (other
// streams, or other threads) race on the array: serialise them.
#include <mutex>

#include "common.cuh"

#define DCRF_STATIC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_static_scratch[DCRF_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the name
// g_static_scratch is only a host-side stand-in, so the address is asked
// from the runtime once per device (with that device current) and cached.
dcrf_status scratch_on_current_device(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DCRF_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DCRF_E_INVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return DCRF_E_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = (unsigned char *)g_scratch_ptr[dev];
    return DCRF_OK;
}

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

__device__ __forceinline__ float4 sload4(const float *p, int64_t i) { return reinterpret_cast<const float4 *>(p)[i]; }
__device__ __forceinline__ float4 sload4(const __half *p, int64_t i) {
    uint2 raw = reinterpret_cast<const uint2 *>(p)[i];
    float2 a = __half22float2(*reinterpret_cast<__half2 *>(&raw.x));
    float2 b = __half22float2(*reinterpret_cast<__half2 *>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// out[a][c] = s0 * sum_k b_k(a) V[vertex_k(a)][c]
template <typename T>
__global__ void k_static_slice(const T *__restrict__ V, int64_t n, int L, int G, int D1,
                               const int32_t *__restrict__ pvid, const float *__restrict__ pbary, float s0,
                               float *__restrict__ out) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * G) return;
    int64_t a = idx / G;
    int g = (int)(idx - a * G);
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < D1; ++k) {
        int v = pvid[a * D1 + k];
        if (v < 0) continue;
        float w = pbary[a * D1 + k];
        float4 q = sload4(V, (int64_t)v * G + g);
        r.x += w * q.x; r.y += w * q.y; r.z += w * q.z; r.w += w * q.w;
    }
    float vals[4] = {r.x, r.y, r.z, r.w};
    for (int i = 0; i < 4; ++i) {
        int c = 4 * g + i;
        if (c < L) out[a * L + c] = s0 * vals[i];
    }
}

}  // namespace

extern "C" size_t dcrf_filter_static_capacity(void) { return DCRF_STATIC_SCRATCH_BYTES; }

extern "C" dcrf_status dcrf_filter_static(dcrf_lattice lat, const float *Y, int L, float *out, int storage,
                                          dcrf_stream stream) {
    if (!lat || !Y || !out || Y == out || L < 1 || L > DCRF_MAX_L) return DCRF_E_INVAL;
    if (storage != DCRF_STORAGE_F32 && storage != DCRF_STORAGE_F16) return DCRF_E_INVAL;
    if (lat->n == 0) return DCRF_OK;
    const int Lp = dcrf_round4(L);
    const size_t esz = storage == DCRF_STORAGE_F16 ? 2 : 4;
    const size_t v_bytes = round256((size_t)lat->m * Lp * sizeof(float));
    const size_t b_bytes = round256((size_t)lat->m * Lp * esz);
    if (v_bytes + 2 * b_bytes > DCRF_STATIC_SCRATCH_BYTES) return DCRF_E_SCRATCH;
    unsigned char *base = nullptr;
    DCRF_CHECK_STATUS(scratch_on_current_device(&base));
    cudaStream_t s = (cudaStream_t)stream;
    float *V = (float *)base;
    void *dst = base + v_bytes;
    void *tmp = base + v_bytes + b_bytes;
    DCRF_TRY(cudaMemsetAsync(V, 0, (size_t)lat->m * Lp * sizeof(float), s));
    DCRF_CHECK_STATUS(dcrf_splat_dense(lat, Y, L, V, Lp, s));
    DCRF_CHECK_STATUS(dcrf_blur(lat, V, dst, tmp, Lp, storage, false, s));
    const int G = Lp / 4;
    const unsigned nb = (unsigned)((lat->n * G + 255) / 256);
    if (storage == DCRF_STORAGE_F16)
        k_static_slice<__half><<<nb, 256, 0, s>>>((const __half *)dst, lat->n, L, G, lat->d + 1, lat->pvid,
                                                  lat->pbary, (float)lat->s0, out);
    else
        k_static_slice<float><<<nb, 256, 0, s>>>((const float *)dst, lat->n, L, G, lat->d + 1, lat->pvid,
                                                 lat->pbary, (float)lat->s0, out);
    DCRF_LAUNCHED();
    return DCRF_OK;
}
