// cdfci_column_noalloc: the get_column operation for callers that cannot
// allocate device memory (for example code running under a memory pool or
// allocator it does not own, or inside a framework that forbids cudaMalloc on
// its hot path).  The caller passes the integrals and the output buffers in
// device memory; every scratch buffer the computation needs lives in the
// file-scope array below, which is part of the library image.
//
// Scratch layout (kScratchBytes in total, shared by every call on a device):
//   [0, 8)                  compaction counter (cleared by every call)
//   [256, 256 + 2*63*63*8)  J and K tables for up to 63 orbitals
//   then                    four pair tables of up to C(63,2) uint16 entries
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/cdfci.h"
#include "cdfci_internal.cuh"
#include "cdfci_kernels.h"

namespace cdfci {
namespace {

constexpr int kNoallocMaxN = kMaxN;                       // 63 spatial orbitals
constexpr size_t kJKBytes = 2ull * kNoallocMaxN * kNoallocMaxN * sizeof(double);
constexpr size_t kPairsOffset = 256 + ((kJKBytes + 255) / 256) * 256;
constexpr size_t kPairsBytes = 4ull * kMaxPairs * sizeof(unsigned short);
constexpr size_t kScratchBytes = kPairsOffset + ((kPairsBytes + 255) / 256) * 256;   // about 80 KB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch on each device (the host-side symbol is a
// stand-in, not a device address).
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int nfail(int code, const char *fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error_message(buf);     // reported by cdfci_last_error()
    return code;
}

long long nbinom(int n, int k) {
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// J_pq = (pp|qq), K_pq = (pq|qp) and the four (i < j) pair tables, written
// into the scratch array; everything the column kernel reads besides h and g.
__global__ void k_noalloc_tables(const double *g, int N, int na, int nb, double *J, double *K,
                                 unsigned short *pairs, int off_ob, int off_va, int off_vb) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * N; t += gridDim.x * blockDim.x) {
        int p = t / N, q = t % N;
        J[t] = g[(((size_t)p * N + p) * N + q) * N + q];
        K[t] = g[(((size_t)p * N + q) * N + q) * N + p];
    }
    const int sizes[4] = {na, nb, N - na, N - nb};
    const int offs[4] = {0, off_ob, off_va, off_vb};
    for (int list = 0; list < 4; ++list) {
        const int n = sizes[list];
        const int cnt = n * (n - 1) / 2;
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
            // t enumerates (i < j) in the order j = 1.., i = 0..j-1
            int j = 1;
            while ((j + 1) * j / 2 <= t) ++j;
            int i = t - j * (j - 1) / 2;
            pairs[offs[list] + t] = (unsigned short)(i | (j << 8));
        }
    }
}

unsigned char *scratch_for_current_device(int *err) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        *err = nfail(CDFCI_ERR_CUDA, "cdfci_column_noalloc: no current CUDA device");
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            *err = nfail(CDFCI_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
            return nullptr;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    return g_scratch_ptr[dev];
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace cdfci

using namespace cdfci;

extern "C" __attribute__((visibility("default"))) int cdfci_column_noalloc(
    const double *h, const double *g, int N, int n_alpha, int n_beta, const uint64_t *key, uint64_t *keys_out,
    double *vals_out, int64_t cap, int64_t *n_out, void *cuda_stream) {
    if (!h || !g || !key || !n_out || (cap > 0 && (!keys_out || !vals_out)))
        return nfail(CDFCI_ERR_ARG, "cdfci_column_noalloc: NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the call waits on the stream (key and count read back), which a capturing
    // stream does not allow: refuse before anything is queued on it
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &cs);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return nfail(CDFCI_ERR_ARG, "cdfci_column_noalloc: stream state unavailable (%s)", cudaGetErrorString(ce));
    }
    if (cs != cudaStreamCaptureStatusNone)
        return nfail(CDFCI_ERR_ARG, "cdfci_column_noalloc: the stream is being captured; this call waits on it");
    if (N < 1 || N > kNoallocMaxN)
        return nfail(CDFCI_ERR_ARG, "cdfci_column_noalloc: N = %d exceeds the scratch limit of %d orbitals", N,
                     kNoallocMaxN);
    if (n_alpha < 0 || n_beta < 0 || n_alpha > N || n_beta > N || n_alpha + n_beta == 0)
        return nfail(CDFCI_ERR_ARG, "cdfci_column_noalloc: electron counts (%d, %d) invalid for N = %d", n_alpha,
                     n_beta, N);
    if (cap < 0) return nfail(CDFCI_ERR_ARG, "cdfci_column_noalloc: cap < 0");
    if (!on_device(h) || !on_device(g) || (cap > 0 && (!on_device(keys_out) || !on_device(vals_out))))
        return nfail(CDFCI_ERR_ARG, "cdfci_column_noalloc: h, g and the outputs must be device memory");
    uint64_t k[2];
    if (cudaMemcpyAsync(k, key, sizeof(k), cudaMemcpyDefault, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return nfail(CDFCI_ERR_CUDA, "cdfci_column_noalloc: reading the key failed");
    const unsigned long long full = (1ull << N) - 1ull;
    if ((k[0] & ~full) || (k[1] & ~full) || __builtin_popcountll(k[0]) != n_alpha || __builtin_popcountll(k[1]) != n_beta)
        return nfail(CDFCI_ERR_ARG, "cdfci_column_noalloc: key does not match N, n_alpha, n_beta");

    int err = 0;
    unsigned char *base = scratch_for_current_device(&err);
    if (!base) return err;
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(base);
    double *J = reinterpret_cast<double *>(base + 256);
    double *K = J + (size_t)N * N;
    unsigned short *pairs = reinterpret_cast<unsigned short *>(base + kPairsOffset);

    Problem P;
    memset(&P, 0, sizeof(P));
    P.N = N; P.na = n_alpha; P.nb = n_beta; P.va = N - n_alpha; P.vb = N - n_beta;
    P.ca2 = (int)nbinom(P.na, 2); P.cb2 = (int)nbinom(P.nb, 2);
    P.cva2 = (int)nbinom(P.va, 2); P.cvb2 = (int)nbinom(P.vb, 2);
    P.seg[0] = 1;
    P.seg[1] = P.seg[0] + (long long)P.na * P.va;
    P.seg[2] = P.seg[1] + (long long)P.nb * P.vb;
    P.seg[3] = P.seg[2] + (long long)P.ca2 * P.cva2;
    P.seg[4] = P.seg[3] + (long long)P.cb2 * P.cvb2;
    P.seg[5] = P.seg[4] + (long long)P.na * P.va * P.nb * P.vb;
    P.mg_va = fdiv_magic((unsigned)P.va); P.mg_vb = fdiv_magic((unsigned)P.vb);
    P.mg_nsb = fdiv_magic((unsigned)(P.nb * P.vb));
    P.mg_cva2 = fdiv_magic((unsigned)P.cva2); P.mg_cvb2 = fdiv_magic((unsigned)P.cvb2);
    P.nh = P.seg[5];
    P.h = h; P.g = g; P.J = J; P.K = K;
    P.pair_oa = pairs;
    P.pair_ob = P.pair_oa + P.ca2;
    P.pair_va = P.pair_ob + P.cb2;
    P.pair_vb = P.pair_va + P.cva2;

    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        k_noalloc_tables<<<8, 256, 0, s>>>(g, N, n_alpha, n_beta, J, K, pairs, P.ca2, P.ca2 + P.cb2,
                                           P.ca2 + P.cb2 + P.cva2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_column(P, k[0], k[1], reinterpret_cast<unsigned long long *>(keys_out), vals_out, cap, counter, s);
    unsigned long long n = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, counter, sizeof(n), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return nfail(CDFCI_ERR_CUDA, "cdfci_column_noalloc: %s", cudaGetErrorString(e));
    *n_out = (int64_t)n;
    if ((int64_t)n > cap)
        return nfail(CDFCI_ERR_CAPACITY, "cdfci_column_noalloc: column has %lld entries, cap is %lld", (long long)n,
                     (long long)cap);
    return CDFCI_OK;
}
