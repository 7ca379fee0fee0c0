// gsr_aprod1_norm_noalloc: the LSQR form of aprod 1 (y = A x + cy y and
// ||y||_2) for callers that cannot allocate device memory -- for example
// code that runs while another component owns the whole device-memory
// budget through its own pool, or a host path where a cudaMalloc would
// synchronise the device at the wrong moment.  Its scratch (the per-block
// partial sums of the norm, the ticket counter and the result slot) lives in
// one file-scope device array instead of memory the library allocates.
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

// Every GPU that loads the library holds these 36 KiB until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

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
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GSR_ERR_CUDA;
        }
        g_scratch_dev[dev] = (unsigned char *)p;
    }
    *out = g_scratch_dev[dev];
    return GSR_OK;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int gsr_aprod1_norm_noalloc(void *hv, const double *x, double *y, double cy,
                                       double *ynorm, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !x || !y || !ynorm)
        return GSR_ERR_ARG;
    // host vectors would need staging memory: only device vectors are taken
    if (!is_device_ptr(x) || !is_device_ptr(y))
        return GSR_ERR_ARG;
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
    rc = scratch_for(h->device, &base);
    if (rc == GSR_OK) {
        SolveState *slot = (SolveState *)base;
        double *partial = (double *)(base + kPartialOff);
        unsigned *counter = (unsigned *)(base + kCounterOff);
        cudaError_t e = cudaMemcpyAsync(&slot->cy, &cy, sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
        if (e == cudaSuccess)
            e = launch_aprod1_with_slots(h, x, y, slot, partial, counter, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ynorm, &slot->beta_new, sizeof(double), cudaMemcpyDefault, st);
        if (e == cudaSuccess && !is_device_ptr(ynorm))
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
