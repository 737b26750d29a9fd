// dcrf_qp_fw_host: the whole QP path for a batch of images held in host
// memory, in one call.
//
// Steps, all on the caller's stream except the bulk uploads:
//   1. upload the RGB images (small: 12 bytes a pixel);
//   2. features (Eq. 4 in kernel form) and the bilateral and spatial
//      lattices (Section 3), whose builds read counts back to the host;
//   3. meanwhile, once the images have landed, a second stream uploads the
//      unaries and y0 (8L bytes a pixel, the bulk of the input), so the copy
//      engine works while the lattices are built;
//   4. Frank-Wolfe (Algorithm 1 with the closed-form step of Appendix B),
//      once both uploads have landed;
//   5. download y and synchronise.
// With pageable host memory the uploads still work but no longer overlap.
#include <chrono>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"

namespace {

struct StreamGuard {
    cudaStream_t s = nullptr;
    ~StreamGuard() {
        if (s) {
            cudaStreamSynchronize(s);   // no upload may outlive the buffers it writes
            cudaStreamDestroy(s);
        }
    }
};

struct EventGuard {
    cudaEvent_t e = nullptr;
    ~EventGuard() {
        if (e) cudaEventDestroy(e);
    }
};

// DCRF_HOST_LOG=1: CUDA events at the phase boundaries, printed to stderr
// as milliseconds after the call's start once the call has synchronised,
// beside the host clock when each mark was issued.
struct PhaseLog {
    static constexpr int kMax = 8;
    bool on = false;
    int n = 0;
    cudaEvent_t ev[kMax] = {};
    const char *name[kMax] = {};
    double host_ms[kMax] = {};
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    PhaseLog() {
        const char *e = std::getenv("DCRF_HOST_LOG");
        on = e && e[0] == '1';
    }
    double host_now() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    void mark(const char *what, cudaStream_t st) {
        if (!on || n >= kMax) return;
        if (cudaEventCreate(&ev[n]) != cudaSuccess) return;
        cudaEventRecord(ev[n], st);
        host_ms[n] = host_now();
        name[n++] = what;
    }
    void print() {
        for (int i = 1; i < n; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[i]);
            std::fprintf(stderr, "dcrf host: %-22s %8.3f ms (issued at host %8.3f ms)\n", name[i], ms, host_ms[i]);
        }
        if (on) std::fprintf(stderr, "dcrf host: %-22s host %8.3f ms (first mark at %.3f)\n", "synchronised", host_now(),
                             host_ms[0]);
    }
    ~PhaseLog() {
        for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
    }
};

struct LatticeGuard {
    dcrf_lattice l[2] = {nullptr, nullptr};
    ~LatticeGuard() {
        for (dcrf_lattice x : l)
            if (x) dcrf_lattice_destroy(x);
    }
};

}  // namespace

extern "C" dcrf_status dcrf_qp_fw_host(const float *rgb, const float *unaries, const float *Y0, float *Y,
                                       const int32_t *widths, const int32_t *heights, int batch, int L,
                                       float theta_alpha, float theta_beta, float theta_gamma,
                                       const float *weights, const float *compat, int iters,
                                       dcrf_fw_record *records, int storage, dcrf_stream stream) {
    if (!widths || !heights || !weights || batch < 1 || L < 1 || L > DCRF_MAX_L || iters < 0) return DCRF_E_INVAL;
    std::vector<int64_t> off(batch + 1, 0);
    for (int b = 0; b < batch; ++b) {
        if (widths[b] < 0 || heights[b] < 0) return DCRF_E_INVAL;
        off[b + 1] = off[b] + (int64_t)widths[b] * heights[b];
    }
    const int64_t n = off[batch];
    if (n > 0 && (!rgb || !unaries || !Y0 || !Y)) return DCRF_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;

    // declared in this order so that, on every return, the upload stream is
    // drained and the lattices destroyed before the scratch is released
    Scratch sc(s);
    LatticeGuard lg;
    EventGuard ready, landed;
    StreamGuard up;
    PhaseLog log;
    log.mark("start", s);

    const size_t nn = (size_t)(n > 0 ? n : 1);
    float *rgb_d, *fb, *fs, *phi_d, *y_d;
    DCRF_CHECK_STATUS(sc.get(&rgb_d, nn * 3));
    DCRF_CHECK_STATUS(sc.get(&fb, nn * 5));
    DCRF_CHECK_STATUS(sc.get(&fs, nn * 2));
    DCRF_CHECK_STATUS(sc.get(&phi_d, nn * L));
    DCRF_CHECK_STATUS(sc.get(&y_d, nn * L));
    DCRF_TRY(cudaEventCreateWithFlags(&ready.e, cudaEventDisableTiming));
    DCRF_TRY(cudaEventCreateWithFlags(&landed.e, cudaEventDisableTiming));
    DCRF_TRY(cudaStreamCreateWithFlags(&up.s, cudaStreamNonBlocking));

    // the images go first: copies in one direction share the copy engine, and
    // the builds wait for the images only.  The upload stream starts once the
    // buffers exist (stream-ordered allocation on s) and the images have landed.
    if (n > 0) DCRF_TRY(cudaMemcpyAsync(rgb_d, rgb, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice, s));
    log.mark("rgb uploaded", s);
    DCRF_TRY(cudaEventRecord(ready.e, s));
    DCRF_TRY(cudaStreamWaitEvent(up.s, ready.e, 0));
    if (n > 0) {
        DCRF_TRY(cudaMemcpyAsync(phi_d, unaries, (size_t)n * L * sizeof(float), cudaMemcpyHostToDevice, up.s));
        DCRF_TRY(cudaMemcpyAsync(y_d, Y0, (size_t)n * L * sizeof(float), cudaMemcpyHostToDevice, up.s));
    }
    DCRF_TRY(cudaEventRecord(landed.e, up.s));
    log.mark("unaries+y0 uploaded", up.s);

    DCRF_CHECK_STATUS(dcrf_features(rgb_d, widths, heights, batch, theta_alpha, theta_beta, theta_gamma, fb, fs,
                                    stream));
    DCRF_CHECK_STATUS(dcrf_lattice_build_batch(fb, off.data(), batch, 5, stream, &lg.l[0]));
    DCRF_CHECK_STATUS(dcrf_lattice_build_batch(fs, off.data(), batch, 2, stream, &lg.l[1]));
    log.mark("lattices built", s);

    DCRF_TRY(cudaStreamWaitEvent(s, landed.e, 0));
    log.mark("solver starts", s);
    DCRF_CHECK_STATUS(dcrf_qp_fw(phi_d, lg.l, weights, 2, compat, L, iters, y_d, records, storage, stream));
    log.mark("solver done", s);
    if (n > 0) DCRF_TRY(cudaMemcpyAsync(Y, y_d, (size_t)n * L * sizeof(float), cudaMemcpyDeviceToHost, s));
    log.mark("y downloaded", s);
    DCRF_TRY(cudaStreamSynchronize(s));
    log.print();
    return DCRF_OK;
}
