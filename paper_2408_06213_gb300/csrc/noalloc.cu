// noalloc.cu -- a shuffle entry point that allocates no device memory.
//
// brr_shuffle keeps its reservation words, pending lists and swap indices in
// scratch that a context grows with cudaMalloc.  Some callers cannot allocate
// device memory on demand: code whose device memory is owned by another
// allocator or capped by a fixed budget, and latency-critical loops that
// cannot afford the device-wide synchronisation cudaMalloc / cudaFree may
// imply.  For them, brr_shuffle_noalloc runs the same kernels with the
// scratch taken from the fixed-size array below, which every device that
// loads this library holds until the process exits.
#include <mutex>

#include "brr_common.cuh"
#include "internal.h"

namespace {

// Reservation words, two pending-pair lists, swap indices and control words
// for BRR_NOALLOC_MAX_N positions (24 bytes each), plus a last 256-byte line
// whose first word is the device error word of the call.
constexpr size_t kNoAllocShuffleBytes = (size_t)BRR_NOALLOC_MAX_N * 24 + 4096;
constexpr size_t kNoAllocBytes = kNoAllocShuffleBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch
    int num_sms = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: look up the device address of
// the scratch array (in host code its name is only a host-side stand-in).
// The address is cached for the life of the process, so a device reset after
// the first call is not supported (the module could reload elsewhere).
brr_status setup_current_device(DeviceSetup &out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return BRR_ENODEV;
    }
    if (dev < 0 || dev >= kMaxDevices) return BRR_ENODEV;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (s.base == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return BRR_ECUDA;
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || sms <= 0) {
            cudaGetLastError();
            return BRR_ECUDA;
        }
        s.base = static_cast<unsigned char *>(p);
        s.num_sms = sms;
    }
    out = s;
    return BRR_OK;
}

}  // namespace

extern "C" brr_status brr_shuffle_noalloc(void *data_dev, uint64_t n, uint32_t elem_bytes,
                                          uint64_t seed, const brr_schedule *sched,
                                          uint32_t *j_out_dev, int *status_dev,
                                          brr_stream_t stream) {
    brr_schedule tmp;
    if (!sched) {
        brr_schedule_paper(&tmp);
        sched = &tmp;
    }
    if (elem_bytes != 4 && elem_bytes != 8) return BRR_EINVAL;
    if (n > BRR_NOALLOC_MAX_N) return BRR_EINVAL;  // larger shuffles need brr_shuffle
    if (!brr::sched_valid(sched->n_k, sched->k_max)) return BRR_EINVAL;
    if (n > 1 && !data_dev) return BRR_EINVAL;
    if (brr::shuffle_scratch_size(n, j_out_dev == nullptr) > kNoAllocShuffleBytes) return BRR_EINVAL;
    DeviceSetup dev;
    brr_status st = setup_current_device(dev);
    if (st != BRR_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int *err = reinterpret_cast<int *>(dev.base + kNoAllocShuffleBytes);
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e != cudaSuccess) return brr::cuda_status(e);
    st = brr::launch_shuffle_on_scratch(data_dev, n, elem_bytes, seed, sched, j_out_dev, dev.base, err,
                                        dev.num_sms, s);
    if (st != BRR_OK) return st;
    if (status_dev) {
        e = cudaMemcpyAsync(status_dev, err, sizeof(int), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return brr::cuda_status(e);
    }
    return BRR_OK;
}
