// OptOrbFCI (Algorithm 4, Sec. "Optimal Orbital Selections"): device kernels of
// the orbital subproblem.  Every array is FP64 and row-major; U is M x N with
// orthonormal columns, the integrals h (M x M) and g (M^4, chemists' order) are
// in the large basis, the RDMs (N x N, N^4) in the small one.
//   k_oo_contract   out[a][n][b] = sum_m in[a][m][b] U[m][n] (one index of a tensor)
//   k_oo_grad       G = 2 (h U) gamma + 2 sum_bcd g''_pbcd Gamma_abcd
//   k_oo_dot        sum_i x_i y_i in a fixed order (one block)
//   k_oo_axpy       y = x - t z
//   k_oo_gram       X^T X (N x N)
//   k_oo_ns         X <- X (3 I - X^T X) / 2 (Newton-Schulz step to the polar factor)
#include <algorithm>

#include "cdfci_internal.cuh"
#include "cdfci_kernels.h"

namespace cdfci {

__global__ void k_oo_contract(const double *in, const double *U, double *out, long long A, int M, int N, long long B) {
    const long long total = A * N * B;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i % B;
        const int n = (int)((i / B) % N);
        const long long a = i / (B * N);
        double s = 0.0;
        for (int m = 0; m < M; ++m) s = fma(in[(a * M + m) * B + b], U[m * N + n], s);
        out[i] = s;
    }
}

__global__ void k_oo_grad(const double *hU, const double *g1, const double *g3, const double *g2, double *G, int M,
                          int N) {
    const int n3 = N * N * N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M * N; i += gridDim.x * blockDim.x) {
        const int p = i / N, a = i - p * N;
        double s1 = 0.0, s2 = 0.0;
        for (int b = 0; b < N; ++b) s1 = fma(hU[p * N + b], g1[b * N + a], s1);
        const double *x = g3 + (size_t)p * n3, *y = g2 + (size_t)a * n3;
        for (int t = 0; t < n3; ++t) s2 = fma(x[t], y[t], s2);
        G[i] = 2.0 * s1 + 2.0 * s2;
    }
}

// one block of 256 threads: strided partial sums, then a fixed tree
__global__ void k_oo_dot(const double *x, const double *y, long long n, double *out) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], y[i], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_oo_axpy(const double *x, const double *z, double t, double *y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] - t * z[i];
}

__global__ void k_oo_scale(double *x, const double *s, long long n) {
    const double f = *s > 0.0 ? 1.0 / sqrt(*s) : 1.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= f;
}

__global__ void k_oo_gram(const double *X, double *Gm, int M, int N) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * N; i += gridDim.x * blockDim.x) {
        const int a = i / N, b = i - a * N;
        double s = 0.0;
        for (int p = 0; p < M; ++p) s = fma(X[p * N + a], X[p * N + b], s);
        Gm[i] = s;
    }
}

__global__ void k_oo_ns(const double *X, const double *Gm, double *Xn, int M, int N) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M * N; i += gridDim.x * blockDim.x) {
        const int p = i / N, a = i - p * N;
        double s = 0.0;
        for (int b = 0; b < N; ++b) s = fma(X[p * N + b], Gm[b * N + a], s);
        Xn[i] = 0.5 * (3.0 * X[i] - s);
    }
}

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
static int oo_grid(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8)); }

cudaError_t oo_contract(const double *in, const double *U, double *out, long long A, int M, int N, long long B,
                        cudaStream_t s) {
    k_oo_contract<<<oo_grid(A * N * B), 256, 0, s>>>(in, U, out, A, M, N, B);
    return cudaGetLastError();
}
cudaError_t oo_grad(const double *hU, const double *g1, const double *g3, const double *g2, double *G, int M, int N,
                    cudaStream_t s) {
    k_oo_grad<<<oo_grid((long long)M * N), 256, 0, s>>>(hU, g1, g3, g2, G, M, N);
    return cudaGetLastError();
}
cudaError_t oo_dot(const double *x, const double *y, long long n, double *out, cudaStream_t s) {
    k_oo_dot<<<1, 256, 0, s>>>(x, y, n, out);
    return cudaGetLastError();
}
cudaError_t oo_axpy(const double *x, const double *z, double t, double *y, long long n, cudaStream_t s) {
    k_oo_axpy<<<oo_grid(n), 256, 0, s>>>(x, z, t, y, n);
    return cudaGetLastError();
}
cudaError_t oo_scale(double *x, const double *sq, long long n, cudaStream_t s) {
    k_oo_scale<<<oo_grid(n), 256, 0, s>>>(x, sq, n);
    return cudaGetLastError();
}
cudaError_t oo_gram(const double *X, double *Gm, int M, int N, cudaStream_t s) {
    k_oo_gram<<<oo_grid((long long)N * N), 256, 0, s>>>(X, Gm, M, N);
    return cudaGetLastError();
}
cudaError_t oo_ns(const double *X, const double *Gm, double *Xn, int M, int N, cudaStream_t s) {
    k_oo_ns<<<oo_grid((long long)M * N), 256, 0, s>>>(X, Gm, Xn, M, N);
    return cudaGetLastError();
}

}  // namespace cdfci
