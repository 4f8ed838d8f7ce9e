// sigkernel_pairs_noalloc: the pairs entry point for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where they need a
// kernel value: code running under an allocator that forbids new device allocations, plugins
// whose host application owns all device memory, or latency-critical loops that must not risk an
// allocation.  For them this file keeps a fixed scratch array in device global memory, sized
// once at library load, and passes it to the ordinary sigkernel_pairs as its workspace.
//
// Facts a user of this entry point needs:
//   * Every GPU that loads the library holds kScratchBytes (64 MiB) of device memory for this
//     array until the process exits.
//   * A call whose workspace need (sigkernel_workspace_size for SK_OP_PAIRS) exceeds
//     kScratchBytes is rejected with SK_ERR_WORKSPACE and a message giving both sizes.
//   * All calls on a device share the one array, which keeps the previous call's contents.  The
//     parts that must start at zero (the work-queue counter and the ordering histogram) are
//     cleared by every call on its stream.  Two calls that overlap on the GPU (different streams
//     without ordering between them) race on the array and give undefined results.
//   * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
//     that device current.  Make that first call before any stream capture on the device.
//   * The call allocates nothing: no cudaMalloc, cudaMallocAsync, cudaFree or allocating library
//     routine runs in it.
// The paper has no counterpart: this is a deployment facility of the library.
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/sigkernel.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;

// The scratch itself.  In host code `g_noalloc_scratch` names a host-side stand-in, not a device
// address; its device address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[64] = {nullptr};
thread_local std::string t_msg;

int set_error(int code, const char* msg) {
    t_msg = msg;
    return code;
}

}  // namespace

extern "C" {

const char* sigkernel_noalloc_last_error(void) { return t_msg.c_str(); }

size_t sigkernel_noalloc_capacity(void) { return kScratchBytes; }

int sigkernel_pairs_noalloc(const sk_paths* X, const sk_paths* Y, int32_t d, int32_t dtype,
                            const int64_t* pair_a, const int64_t* pair_b, int64_t npairs,
                            const sk_options* opt, double* out, void* stream) {
    t_msg.clear();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return set_error(SK_ERR_CUDA, "sigkernel_pairs_noalloc: no usable current device");
    void* addr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                char buf[256];
                snprintf(buf, sizeof(buf), "sigkernel_pairs_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                return set_error(SK_ERR_CUDA, buf);
            }
            g_addr[dev] = p;
        }
        addr = g_addr[dev];
    }
    size_t need = 0;
    int rc = sigkernel_workspace_size(SK_OP_PAIRS, X, Y, d, npairs, opt, &need);
    if (rc != SK_OK) return set_error(rc, sigkernel_last_error());
    if (need > kScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "sigkernel_pairs_noalloc: this call needs %zu bytes of scratch, more than the fixed %zu",
                 need, kScratchBytes);
        return set_error(SK_ERR_WORKSPACE, buf);
    }
    rc = sigkernel_pairs(X, Y, d, dtype, pair_a, pair_b, npairs, opt, out, addr, kScratchBytes, stream);
    if (rc != SK_OK) return set_error(rc, sigkernel_last_error());
    return SK_OK;
}

}  // extern "C"
