// cdfci_probe_slots: the memory system's rate for the hash scatter's access
// pattern, measured on the device that runs it.  Each operation takes one
// pseudo-random 32-byte slot of a table larger than L2 and does what the
// scatter's lookup of an existing key does there: one 32-byte load of the slot
// {A, B, c, b} and a fire-and-forget FP64 add to b.
// Slots are independent of one another, so every lane keeps kProbeU
// operations in flight: the rate is the ceiling for random 32-byte slot
// read-modify-write traffic, not the rate of a dependent probe chain.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/cdfci.h"
#include "cdfci_internal.cuh"
#include "cdfci_kernels.h"

namespace cdfci {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeU = 8;                 // operations in flight per lane

__global__ void __launch_bounds__(kProbeThreads) k_probe_slots(Slot *t, unsigned long long mask, long long n_ops,
                                                               unsigned long long seed, double *sink) {
    const long long nt = (long long)gridDim.x * blockDim.x;
    long long op = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * kProbeU;
    double acc = 0.0;
    for (; op < n_ops; op += nt * kProbeU) {
        unsigned long long s[kProbeU], ka[kProbeU], kb[kProbeU], cb[kProbeU], bb[kProbeU];
#pragma unroll
        for (int u = 0; u < kProbeU; ++u) s[u] = mix64(seed + (unsigned long long)(op + u)) & mask;
#pragma unroll
        for (int u = 0; u < kProbeU; ++u) {
            if (op + u < n_ops)
                asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
                             : "=l"(ka[u]), "=l"(kb[u]), "=l"(cb[u]), "=l"(bb[u])
                             : "l"(t + s[u]));
        }
#pragma unroll
        for (int u = 0; u < kProbeU; ++u) {
            if (op + u < n_ops) {
                // the add depends on the key's load, as a lookup's does
                atomicAdd(&t[s[u]].bv, (ka[u] ^ kb[u]) == 1ull ? 2.0 : 1.0);
                acc += __longlong_as_double((long long)cb[u]);
            }
        }
    }
    if (acc == -1.0) *sink = acc;          // keeps the c loads
}

}  // namespace
}  // namespace cdfci

using namespace cdfci;

extern "C" __attribute__((visibility("default"))) int cdfci_probe_slots(void *table, int log2_slots, int64_t n_ops,
                                                                       uint64_t seed, void *cuda_stream) {
    if (!table || log2_slots < 10 || log2_slots > 34 || n_ops < 0) {
        set_last_error_message("cdfci_probe_slots: NULL table, log2_slots outside [10, 34] or n_ops < 0");
        return CDFCI_ERR_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(table) & 31u) != 0) {
        set_last_error_message("cdfci_probe_slots: the table must be 32-byte aligned");
        return CDFCI_ERR_ARG;
    }
    if (n_ops == 0) return CDFCI_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_probe_slots, kProbeThreads, 0) != cudaSuccess) {
        set_last_error_message("cdfci_probe_slots: device query failed");
        return CDFCI_ERR_CUDA;
    }
    const long long need = (n_ops + (long long)kProbeThreads * kProbeU - 1) / ((long long)kProbeThreads * kProbeU);
    const int grid = (int)(need < (long long)sms * per ? need : (long long)sms * per);
    // the sink is never written for finite c (acc == -1 is not reached with the bench's table);
    // it points into the table's first slot so that no allocation is needed
    double *sink = &static_cast<Slot *>(table)->bv;
    k_probe_slots<<<grid, kProbeThreads, 0, s>>>(static_cast<Slot *>(table), (1ull << log2_slots) - 1ull, n_ops,
                                                 seed, sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error_message(cudaGetErrorString(e));
        return CDFCI_ERR_CUDA;
    }
    return CDFCI_OK;
}
