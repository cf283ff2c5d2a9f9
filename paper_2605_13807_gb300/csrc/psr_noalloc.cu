// psr_logpsi_noalloc: log psi without any device allocation.
//
// Some callers cannot call cudaMalloc: a host program whose device memory is
// owned entirely by another runtime's pool (a direct cudaMalloc would fail or
// fragment that pool), a latency-critical loop that cannot afford the
// implicit synchronisation an allocation may cause, or a sandboxed plug-in
// that is not given the allocation API at all.  This entry point serves them:
// it runs the same kernels as psr_logpsi, but every byte of scratch (packed
// weights, bit-packed spins, the job counter and a status word) lives in the
// fixed array below, which CUDA reserves on each device when the library's
// module is loaded there and keeps until the process exits.
//
// Set-up: the first call made on a device, with that device current, looks up
// the device address of the array with cudaGetSymbolAddress (host code cannot
// use the array's name as a device pointer; that name is only a host-side
// stand-in) and the SM count; later calls on that device reuse them.  That
// first call should be made before any stream capture begins.
//
// Sharing: all calls in the process share the one array per device and it
// keeps whatever the last call left in it; each call clears the job counter
// and the status word itself before use.  Two calls whose work overlaps on a
// device (different streams, or different host threads) race on the array.
//
// Status: the kernels record device-side failures (a spin byte other than
// 0/1, an expired bounded wait, a tensor-memory allocation that does not
// start at column 0) in a status word at a fixed place in the array; such a
// call still returns PSR_OK, since it does not wait for its kernels, and may
// leave `out` partly or wholly unwritten.  psr_noalloc_status reads that word
// after the call's work has finished, without allocating.
#include <cuda_runtime.h>

#include <mutex>

#include "psr_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;  // stated maximum: 8 MiB per device
constexpr size_t kBitsBytes = size_t(4) << 20;     // bit-packed spins of one batch of samples
constexpr size_t kOffCounter = kScratchBytes - 512; // job counter (fixed place)
constexpr size_t kOffStatus = kScratchBytes - 256;  // status word (fixed place, read by psr_noalloc_status)
constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_psr_noalloc_scratch[kScratchBytes];

namespace {

using namespace psr;

struct DeviceSetup {
    bool ready = false;
    unsigned char *base = nullptr;  // device address of g_psr_noalloc_scratch
    int num_sms = 1;
};

DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// Once per device, with the device current: device address of the array.
int setup_current_device(DeviceSetup **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PSR_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return PSR_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_psr_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return PSR_ECUDA;
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return PSR_ECUDA;
        }
        s.base = static_cast<unsigned char *>(p);
        s.num_sms = sms > 0 ? sms : 1;
        s.ready = true;
    }
    *out = &s;
    return PSR_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int to_rc(cudaError_t e) { return e == cudaSuccess ? PSR_OK : PSR_ECUDA; }

}  // namespace

extern "C" int psr_logpsi_noalloc(const psr_params *params, const uint8_t *spins, int64_t n,
                                  int32_t L, float *out, void *stream) {
    if (!params || !params->theta || !spins || !out) return PSR_EINVAL;
    const int nL = params->n_layers, H = params->hidden;
    if (nL < 1 || nL > kMaxLayers) return PSR_EINVAL;
    if (H != 32 && H != 64 && H != 128) return PSR_EINVAL;
    if (params->u1_mask != 0 && params->u1_mask != 1) return PSR_EINVAL;
    if (params->precision == PSR_FP16) return PSR_EUNSUPPORTED;
    if (params->precision != PSR_FP32 && params->precision != PSR_BF16) return PSR_EINVAL;
    if (n < 1 || L < 1 || n > ((int64_t)1 << 31)) return PSR_EINVAL;
    if (params->u1_mask && (L % 2)) return PSR_EINVAL;
    const bool bf16 = params->precision == PSR_BF16;
    if (bf16 && (H != 128 || nL != 3)) return PSR_EUNSUPPORTED;

    // Carve-up of the array: packed FP32 weights, BF16 images, bit-packed
    // spins of one batch; the job counter and the status word sit at fixed
    // places at its end.
    const ThetaLayout tl = theta_layout(nL, H);
    const F32Layout fl = f32_layout(nL, H);
    const size_t off_pk = 0;
    const size_t off_pkb = align256(off_pk + (size_t)fl.total * sizeof(float));
    const size_t off_bits = align256(off_pkb + (bf16 ? bf16_packed_bytes() : 0));
    if (off_bits + kBitsBytes > kOffCounter) return PSR_EINVAL;
    const int64_t W = (L + 63) / 64 + 1;
    const int64_t rows_per_batch = (int64_t)(kBitsBytes / ((size_t)W * sizeof(uint64_t)));
    if (rows_per_batch < 1) return PSR_EINVAL;  // one configuration longer than the array allows

    // Only device arrays: staging host arrays would need scratch of size n*L.
    if (!on_device(params->theta) || !on_device(spins) || !on_device(out)) return PSR_EINVAL;

    DeviceSetup *dev = nullptr;
    int rc = setup_current_device(&dev);
    if (rc != PSR_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float *pk = reinterpret_cast<float *>(dev->base + off_pk);
    void *pkb = dev->base + off_pkb;
    uint64_t *bits = reinterpret_cast<uint64_t *>(dev->base + off_bits);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(dev->base + kOffCounter);
    int *status = reinterpret_cast<int *>(dev->base + kOffStatus);

    if ((rc = to_rc(cudaMemsetAsync(status, 0, sizeof(int), st))) != PSR_OK) return rc;
    if ((rc = to_rc(launch_pack_theta_f32(params->theta, tl, fl, pk, st))) != PSR_OK) return rc;
    if (bf16 && (rc = to_rc(launch_pack_theta_bf16(params->theta, tl, pkb, st))) != PSR_OK) return rc;
    for (int64_t first = 0; first < n; first += rows_per_batch) {
        const int64_t cnt = (n - first < rows_per_batch) ? n - first : rows_per_batch;
        if ((rc = to_rc(launch_bitpack(spins + first * L, cnt, L, (int)W, bits, status, st))) != PSR_OK)
            return rc;
        if ((rc = to_rc(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st))) != PSR_OK)
            return rc;
        FwdJobs jb{};
        jb.mode = 0;
        jb.n_groups = 1;
        jb.g[0].u1 = params->u1_mask;
        jb.g[0].N = L;
        jb.g[0].W = (int)W;
        jb.g[0].n_jobs = cnt;
        jb.g[0].bits = bits;
        jb.g[0].out = out + first;
        jb.job_counter = counter;
        jb.status = status;
        rc = to_rc(bf16 ? launch_fwd_bf16(jb, pkb, pk, fl, dev->num_sms, st)
                        : launch_fwd_f32(jb, pk, fl, dev->num_sms, st));
        if (rc != PSR_OK) return rc;
    }
    return PSR_OK;
}

extern "C" int psr_noalloc_status(void *stream) {
    // Waits for the stream, then copies the status word out of the fixed
    // array by its symbol (no address set-up and no allocation needed).
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return PSR_ECUDA;
    }
    int word = 0;
    if (cudaMemcpyFromSymbol(&word, g_psr_noalloc_scratch, sizeof(int), kOffStatus,
                             cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return PSR_ECUDA;
    }
    return word;
}
