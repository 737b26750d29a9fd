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

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// Device address of the array on the device of stream s.  In host code the
// name g_static_scratch is only a host-side stand-in, so the address is asked
// from the runtime once per device, with that device current (made current
// for the lookup when the stream belongs to another one), and cached.
// dcrf_lattice_build calls this too, so that the lookup normally happens
// before any dcrf_filter_static call.
dcrf_status dcrf_static_scratch(cudaStream_t s, unsigned char **out) {
    int dev = 0, cur = 0;
    if (cudaStreamGetDevice(s, &dev) != cudaSuccess || cudaGetDevice(&cur) != cudaSuccess) return DCRF_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DCRF_E_INVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        if (dev != cur && cudaSetDevice(dev) != cudaSuccess) return DCRF_E_CUDA;
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (dev != cur) cudaSetDevice(cur);
        if (e != cudaSuccess || !p) return DCRF_E_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = (unsigned char *)g_scratch_ptr[dev];
    return DCRF_OK;
}

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
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    DCRF_CHECK_STATUS(dcrf_static_scratch(s, &base));
    float *V = (float *)base;
    void *dst = base + v_bytes;
    void *tmp = base + v_bytes + b_bytes;
    DCRF_TRY(cudaMemsetAsync(V, 0, (size_t)lat->m * Lp * sizeof(float), s));
    DCRF_CHECK_STATUS(dcrf_splat_dense(lat, Y, L, V, Lp, s));
    DCRF_CHECK_STATUS(dcrf_blur(lat, V, dst, tmp, Lp, storage, false, s));
    return dcrf_slice(lat, dst, Lp, L, storage, out, s);
}
