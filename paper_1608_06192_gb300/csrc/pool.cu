// The library's own stream-ordered memory pool, one per device.
//
// Every call takes its device scratch with a stream-ordered allocation and
// returns it before it ends.  From the device's default pool, whose release
// threshold is zero, memory freed by one call goes back to the driver at the
// next synchronisation and the next call maps it again (a few milliseconds
// per call at the sizes of a 32-image batch).  This pool keeps what it has
// mapped, like a caching allocator; dcrf_pool_trim hands the unused part
// back.  DCRF_POOL=default selects the default pool instead.  Allocations
// made while the stream is being captured into a graph use the default pool
// (graph memory nodes).
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};
int g_mode = -1;   // 1: own pools, 0: the default pool

}  // namespace

cudaMemPool_t dcrf_scratch_pool(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    int dev = 0;
    if (cudaStreamGetDevice(s, &dev) != cudaSuccess) return nullptr;
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_mode < 0) {
        const char *e = std::getenv("DCRF_POOL");
        g_mode = (e && std::strcmp(e, "default") == 0) ? 0 : 1;
    }
    if (g_mode == 0) return nullptr;
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;
        if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return nullptr;
        }
        g_pool[dev] = p;
    }
    return g_pool[dev];
}

extern "C" dcrf_status dcrf_pool_trim(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (cudaMemPool_t p : g_pool)
        if (p && cudaMemPoolTrimTo(p, 0) != cudaSuccess) return DCRF_E_CUDA;
    return DCRF_OK;
}
