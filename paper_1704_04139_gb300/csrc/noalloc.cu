// noalloc.cu -- FP64 residual with gates taken at u_old, using scratch that
// lives in this module's static device memory instead of the cell's buffers.
//
// Some callers cannot allocate device memory at the moment they need a
// residual: a serving loop whose memory is fully reserved up front by another
// allocator (a cudaMalloc there can fail on a full device or stall while the
// device synchronises), or a latency-bound thread that must not wait on the
// allocator's locks or on a device-wide free.  This entry point needs F bytes
// of gate scratch and takes them from a fixed array in static device memory,
// so its success path calls no allocating routine of CUDA, of this library or
// of any other library.
#include "mb_internal.h"

#include <atomic>

namespace {

// Gate scratch: one byte per plating face.  Nothing in it has to start at
// zero: every byte the residual kernel reads is written by the gate kernel
// earlier on the same stream within the same call.
static __device__ __align__(256) uint8_t g_gate_scratch[MB_NOALLOC_MAX_FACES];

constexpr int MAX_DEVICES = 64;
std::atomic<uint8_t*> g_scratch_addr[MAX_DEVICES];

// Address of the scratch array on device dev (the current device), resolved
// once per device.
int scratch_address(int dev, uint8_t** out) {
    if (dev < 0 || dev >= MAX_DEVICES) {
        ::mb::set_error("mb_residual_dev_noalloc: device index out of range");
        return MB_EINVAL;
    }
    uint8_t* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        void* addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_gate_scratch);
        if (e != cudaSuccess) return ::mb::cuda_fail(e, "cudaGetSymbolAddress(gate scratch)");
        p = static_cast<uint8_t*>(addr);
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return MB_OK;
}

}  // namespace

extern "C" int mb_residual_dev_noalloc(mb_cell* c, const double* u, const double* u_old, double dt, double I_app,
                                       double* r, void* stream) {
    if (!c || !u || !u_old || !r || !(dt > 0)) {
        ::mb::set_error("mb_residual_dev_noalloc: invalid argument");
        return MB_EINVAL;
    }
    if (c->D.F > (int64_t)MB_NOALLOC_MAX_FACES) {
        ::mb::set_error("mb_residual_dev_noalloc: the cell has more plating faces than the static scratch "
                        "holds (MB_NOALLOC_MAX_FACES)");
        return MB_EINVAL;
    }
    // the cell's buffers live on c->device: the scratch address and the
    // launches must be those of that device
    int dev = -1;
    MB_CUDA(cudaGetDevice(&dev));
    if (dev != c->device) {
        ::mb::set_error("mb_residual_dev_noalloc: the current device is not the cell's device");
        return MB_EINVAL;
    }
    uint8_t* gate = nullptr;
    int rc = scratch_address(dev, &gate);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = ::mb::launch_gate_residual_unprofiled(c, u, u_old, gate, dt, I_app, r, s);
    if (rc) return rc;
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
}
