// gsr_aprod1_norm_noalloc: the LSQR form of aprod 1 (y = A x + cy y and
// ||y||_2) for callers that cannot allocate device memory -- for example
// code that runs while another component owns the whole device-memory
// budget through its own pool, or a host path where a cudaMalloc would
// synchronise the device at the wrong moment.  Its scratch (the per-block
// partial sums of the norm, the ticket counter and the result slot) lives in
// one file-scope device array instead of memory the library allocates.
//
// The array's device address is looked up once per device by gsr_create
// (noalloc_prepare), which allocates anyway: under lazy module loading that
// lookup is what makes this file's module, and with it the array, resident
// on the device, so the entry point itself never triggers a module load.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "gsr_internal.cuh"

namespace gsr {
cudaError_t launch_aprod1_with_slots(const gsr_handle_t *h, const double *x, double *y,
                                     SolveState *st_slot, double *partial, unsigned *counter,
                                     cudaStream_t st);
int aprod1_grid_blocks(const gsr_handle_t *h);
}  // namespace gsr

using namespace gsr;

namespace {

// Layout of the static scratch: [0, 256) state slot, then one double per
// thread block (kMaxPartials of them), then the ticket counter.
constexpr size_t kStateBytes = 256;
constexpr size_t kPartialOff = kStateBytes;
constexpr size_t kCounterOff = kPartialOff + sizeof(double) * kMaxPartials;
constexpr size_t kScratchBytes = 36 * 1024;
static_assert(sizeof(SolveState) <= kStateBytes, "state slot too small");
static_assert(kCounterOff + 256 <= kScratchBytes, "scratch too small");

// Every GPU on which a handle has been created holds these 36 KiB until the
// process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Start of a call, on the caller's stream: the coefficient of the old y
// (passed by value, so nothing is copied from host memory) and a cleared
// ticket counter.
__global__ void k_noalloc_begin(SolveState *slot, unsigned *counter, double cy)
{
    if (threadIdx.x == 0) {
        slot->cy = cy;
        *counter = 0u;
    }
}

// Device address of g_noalloc_scratch per device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_dev[kMaxDevices];
std::mutex g_scratch_mu;

int scratch_for(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return GSR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        cudaFuncAttributes fa;
        if (e == cudaSuccess)  // loads the start kernel now as well
            e = cudaFuncGetAttributes(&fa, k_noalloc_begin);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GSR_ERR_CUDA;
        }
        g_scratch_dev[dev] = (unsigned char *)p;
    }
    *out = g_scratch_dev[dev];
    return GSR_OK;
}

// Where a pointer lives, for the handle's device: kOnDevice (device memory
// of that device, or managed memory), kOnHost (pageable or page-locked host
// memory) or kElsewhere (another device's memory, reached only over the peer
// link, or an unknown pointer).
enum PtrKind { kOnDevice, kOnHost, kElsewhere };

PtrKind ptr_kind(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return kElsewhere;
    }
    switch (a.type) {
    case cudaMemoryTypeManaged: return kOnDevice;
    case cudaMemoryTypeDevice: return a.device == dev ? kOnDevice : kElsewhere;
    case cudaMemoryTypeHost:
    case cudaMemoryTypeUnregistered: return kOnHost;
    default: return kElsewhere;
    }
}

}  // namespace

namespace gsr {

// Set-up at handle creation, with the handle's device current: the scratch
// address of this device and the start kernel, resident from now on.
int noalloc_prepare(int dev)
{
    unsigned char *base = nullptr;
    return scratch_for(dev, &base);
}

}  // namespace gsr

extern "C" int gsr_aprod1_norm_noalloc(void *hv, const double *x, double *y, double cy,
                                       double *ynorm, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !x || !y || !ynorm)
        return GSR_ERR_ARG;
    // host vectors would need staging memory, and another device's memory
    // would be reached over the peer link: only the handle's device is taken
    if (ptr_kind(x, h->device) != kOnDevice || ptr_kind(y, h->device) != kOnDevice)
        return GSR_ERR_ARG;
    const PtrKind nk = ptr_kind(ynorm, h->device);
    if (nk == kElsewhere)
        return GSR_ERR_ARG;
    const bool host_norm = nk == kOnHost;
    const int blocks = aprod1_grid_blocks(h);
    if (blocks < 1 || blocks > kMaxPartials)
        return GSR_ERR_ARG;  // more per-block partials than the scratch holds

    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return GSR_ERR_CUDA;
    }
    if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) {
        cudaGetLastError();
        return GSR_ERR_CUDA;
    }
    int rc = GSR_OK;
    unsigned char *base = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    rc = scratch_for(h->device, &base);  // cached by gsr_create
    if (rc == GSR_OK) {
        SolveState *slot = (SolveState *)base;
        double *partial = (double *)(base + kPartialOff);
        unsigned *counter = (unsigned *)(base + kCounterOff);
        k_noalloc_begin<<<1, 32, 0, st>>>(slot, counter, cy);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = launch_aprod1_with_slots(h, x, y, slot, partial, counter, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ynorm, &slot->beta_new, sizeof(double),
                                host_norm ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && host_norm)
            e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = GSR_ERR_CUDA;
        }
    }
    if (cur >= 0 && cur != h->device)
        cudaSetDevice(cur);
    return rc;
}
