// sd_expect_noalloc: the expectation value <psi|O|psi> without any device
// allocation.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed device
// memory budget owned by another allocator (a framework's caching pool, an
// embedded runtime that reserves all memory up front), or a loop that must
// not hit cudaMalloc's implicit device synchronisation.  For them this entry
// point keeps its scratch -- the per-block partial sums of one term and the
// per-term results -- in one file-scope static device array, so it needs no
// allocation at all; the caller passes the state and the observable and
// receives the value.
//
// The array has a fixed size (kScratchBlocks + kScratchTerms + 1 doubles,
// about 41 KB) and every GPU that loads the library holds it until the
// process exits.  All calls share it: a call overwrites what the previous
// call left there (each slot is written before it is read), and calls that
// run at the same time on the GPU -- on different streams, or from
// different host threads -- race on it and give wrong results.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/sd.h"
#include "kernels.cuh"

namespace {

constexpr int kScratchBlocks = 1024;   // partial sums of one term
constexpr int kScratchTerms = 4096;    // one result per observable term
constexpr int kMaxDevices = 64;

struct Scratch {
    double partial[kScratchBlocks];
    double term[kScratchTerms];
    double total;
};

__device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(Scratch)];

std::mutex g_mu;
Scratch *g_addr[kMaxDevices] = {};

// Messages go to the library's last-error slot (sd_last_error(NULL)).
sd_status err(sd_status s, const std::string &m) {
    sd::set_last_error(m);
    return s;
}

// Device address of the scratch array on the current device: looked up once
// per device (with that device current) and cached.
sd_status scratch_for_current_device(Scratch **out, int *num_sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(SD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(SD_EINVAL, "device index out of range");
    e = cudaDeviceGetAttribute(num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return err(SD_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return err(SD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<Scratch *>(p);
    }
    *out = g_addr[dev];
    return SD_OK;
}

}  // namespace

extern "C" sd_status sd_expect_noalloc(int n, const void *d_state, sd_dtype dtype, int64_t mo,
                                       const uint64_t *ox, const uint64_t *oz, const double *oc,
                                       double *out_host, void *cuda_stream) {
    if (n < 1 || n > 40) return err(SD_EINVAL, "n must be in [1, 40]");
    if (!d_state || !out_host) return err(SD_EINVAL, "null state or output pointer");
    if (dtype != SD_C64 && dtype != SD_C128) return err(SD_EINVAL, "dtype must be SD_C64 or SD_C128");
    if (mo < 0 || (mo > 0 && (!ox || !oz || !oc))) return err(SD_EINVAL, "invalid observable arrays");
    if (mo > kScratchTerms)
        return err(SD_EINVAL, "sd_expect_noalloc takes at most " + std::to_string(kScratchTerms) +
                                  " observable terms (fixed scratch size); use sd_expect for more");
    const uint64_t lim = (uint64_t(1) << n) - 1;
    for (int64_t k = 0; k < mo; k++)
        if ((ox[k] & ~lim) || (oz[k] & ~lim) || !std::isfinite(oc[k]))
            return err(SD_EINVAL, "observable term " + std::to_string(k) + " is invalid");
    if (mo == 0) {
        *out_host = 0.0;
        return SD_OK;
    }
    Scratch *S = nullptr;
    int sms = 0;
    sd_status s = scratch_for_current_device(&S, &sms);
    if (s != SD_OK) return s;
    const bool dbl = dtype == SD_C128;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int64_t blocks = (((int64_t)1 << n) + 255) / 256;
    if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
    if (blocks > kScratchBlocks) blocks = kScratchBlocks;
    if (blocks < 1) blocks = 1;
    for (int64_t k = 0; k < mo; k++) {
        // one pass per term writes S->partial[0..blocks); its reduction writes S->term[k]
        cudaError_t e = sd::launch_expect_pauli(dbl, d_state, n, ox[k], oz[k], oc[k], S->partial,
                                                (int)blocks, st);
        if (e == cudaSuccess) e = sd::launch_reduce(S->partial, blocks, S->term + k, 0, st);
        if (e != cudaSuccess) return err(SD_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    cudaError_t e = sd::launch_reduce(S->term, mo, &S->total, 0, st);
    double v = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v, &S->total, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return err(SD_ECUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    *out_host = v;
    return SD_OK;
}
