// Spin-summed reduced density matrices of the stored vector and the energy's
// derivatives (Sec. "Optimal Orbital Selections").
//
//   gamma_pq   = sum_s  <a+_ps a_qs> / c.c
//   Gamma_pqrs = sum_st <a+_ps a+_rt a_st a_qs> / c.c       (chemists' order)
//
// so that E = sum h_pq gamma_pq + 1/2 sum (pq|rs) Gamma_pqrs (Eq. general-ham
// with v_PQRS = (pr|qs)).  For each stored determinant J with c_J != 0 a warp
// walks the excitation list of J with the same decoder as the column kernel
// (all singles and doubles, whatever the value of H), looks each excited
// determinant I up in the table, and adds c_I c_J <I|op|J> to the entries the
// excitation reaches:
//   I = J                 gamma_pp, Gamma_pprr (direct), Gamma_prrp (exchange)
//   single q -> p         gamma_pq; with every other occupied spin-orbital r:
//                         Gamma_pqrr, Gamma_rrpq, and for the same spin
//                         -Gamma_prrq, -Gamma_rqpr
//   double i->a, j->b     Gamma_aibj, Gamma_bjai; same spin also -Gamma_ajbi,
//                         -Gamma_biaj
// The sign <I|a+_a a+_b a_j a_i|J> equals the sign of the sequential
// excitation i->a then j->b that the column decoder returns.  Diagonal-type
// terms go to per-block shared-memory accumulators (a few hot entries), the
// rest to FP64 atomics in global memory.
#include <cuda_runtime.h>

#include "cdfci_internal.cuh"
#include "cdfci_kernels.h"

namespace cdfci {
namespace {

__device__ __forceinline__ int occ_orbital(const ColLists &L, int na, int t) { return t < na ? L.occA[t] : L.occB[t - na]; }

__global__ void __launch_bounds__(256) k_rdm_accumulate(Problem P, IterState *st, double *g1, double *g2,
                                                        double *norm) {
    extern __shared__ double dsh[];                    // N (gamma_pp) + N^2 (Gamma_pprr) + N^2 (Gamma_prrp)
    __shared__ ColLists Lw[8];
    __shared__ double s_norm[8];
    const int N = P.N, N2 = N * N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *d1 = dsh, *dd = dsh + N, *dx = dsh + N + N2;
    for (int t = threadIdx.x; t < N + 2 * N2; t += blockDim.x) dsh[t] = 0.0;
    __syncthreads();
    const long long nh = P.seg[5];                     // every excitation (the RDM does not depend on H)
    const int na = P.na, ne = P.na + P.nb;
    double nrm = 0.0;
    const long long nwarps = (long long)gridDim.x * 8;
    for (long long sl = (long long)blockIdx.x * 8 + warp; sl < P.capacity; sl += nwarps) {
        const Slot S = P.table[sl];
        const unsigned long long A = S.a, B = S.b & kKeyMaskB;
        if ((A | B) == 0ull || S.c == 0.0) continue;    // warp-uniform
        const double cJ = S.c, c2 = cJ * cJ;
        nrm = fma(cJ, cJ, nrm);
        ColLists &L = Lw[warp];
        for (int t = lane; t < N; t += 32) {
            int ra = __popcll(A & low_mask(t)), rb = __popcll(B & low_mask(t));
            if ((A >> t) & 1ull) L.occA[ra] = (unsigned char)t; else L.virA[t - ra] = (unsigned char)t;
            if ((B >> t) & 1ull) L.occB[rb] = (unsigned char)t; else L.virB[t - rb] = (unsigned char)t;
        }
        __syncwarp();
        // I = J: number operators
        for (int t = lane; t < ne; t += 32) atomicAdd(&d1[occ_orbital(L, na, t)], c2);
        for (int t = lane; t < ne * ne; t += 32) {
            const int u = t / ne, v = t - u * ne;
            if (u == v) continue;
            const int p = occ_orbital(L, na, u), r = occ_orbital(L, na, v);
            atomicAdd(&dd[p * N + r], c2);
            if ((u < na) == (v < na)) atomicAdd(&dx[p * N + r], -c2);
        }
        // I = an excitation of J
        for (long long e = 1 + lane; e < nh; e += 32) {
            unsigned long long oa, ob;
            ElemIdx x;
            decode_element(P, L, A, B, e, oa, ob, x);
            bool ins = false;
            const long long s = table_find(P, st, oa, ob, false, &ins);
            if (s < 0) continue;
            const double cI = __ldcg(&P.table[s].c);
            if (cI == 0.0) continue;
            const double v = apply_parity(cI * cJ, x.sgn);
            const int i = x.i, a = x.a;
            if (x.kind <= 1) {                         // single i -> a (spin of kind)
                atomicAdd(&g1[a * N + i], v);
                const int spin = x.kind;               // 0 alpha, 1 beta
                for (int t = 0; t < ne; ++t) {
                    const int ts = t < na ? 0 : 1;
                    const int r = occ_orbital(L, na, t);
                    if (ts == spin && r == i) continue;
                    atomicAdd(&g2[((a * N + i) * N + r) * N + r], v);
                    atomicAdd(&g2[((r * N + r) * N + a) * N + i], v);
                    if (ts == spin) {
                        atomicAdd(&g2[((a * N + r) * N + r) * N + i], -v);
                        atomicAdd(&g2[((r * N + i) * N + a) * N + r], -v);
                    }
                }
            } else {                                   // double i->a, j->b
                const int j = x.j, b = x.b;
                atomicAdd(&g2[((a * N + i) * N + b) * N + j], v);
                atomicAdd(&g2[((b * N + j) * N + a) * N + i], v);
                if (x.kind <= 3) {
                    atomicAdd(&g2[((a * N + j) * N + b) * N + i], -v);
                    atomicAdd(&g2[((b * N + i) * N + a) * N + j], -v);
                }
            }
        }
        __syncwarp();
    }
    // block sums: the shared diagonal accumulators and the norm
    nrm = __shfl_sync(0xffffffffu, nrm, 0);             // lanes of a warp hold the same value
    if (lane == 0) s_norm[warp] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s_norm[w];
        atomicAdd(norm, t);
    }
    for (int t = threadIdx.x; t < N; t += blockDim.x)
        if (d1[t] != 0.0) atomicAdd(&g1[t * N + t], d1[t]);
    for (int t = threadIdx.x; t < N2; t += blockDim.x) {
        const int p = t / N, r = t - p * N;
        if (dd[t] != 0.0) atomicAdd(&g2[((p * N + p) * N + r) * N + r], dd[t]);
        if (dx[t] != 0.0) atomicAdd(&g2[((p * N + r) * N + r) * N + p], dx[t]);
    }
}

// gamma and Gamma divided by c.c, averaged over the symmetries a real
// wavefunction gives them exactly (gamma_pq = gamma_qp; Gamma_pqrs = Gamma_rspq
// = Gamma_qpsr = Gamma_srqp), which removes the rounding asymmetry of the sums.
__global__ void k_rdm_finalize(int N, const double *g1, const double *g2, const double *norm, double *o1, double *o2) {
    const double inv = 1.0 / *norm;
    const int N2 = N * N;
    const long long N4 = (long long)N2 * N2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N4 + N2; t += (long long)gridDim.x * blockDim.x) {
        if (t < N2) {
            const int p = (int)t / N, q = (int)t - p * N;
            o1[t] = 0.5 * (g1[p * N + q] + g1[q * N + p]) * inv;
            continue;
        }
        const long long u = t - N2;
        const int s = (int)(u % N), r = (int)((u / N) % N), q = (int)((u / N2) % N), p = (int)(u / ((long long)N2 * N));
        const double v = (g2[((p * N + q) * N + r) * N + s] + g2[((r * N + s) * N + p) * N + q]) +
                         (g2[((q * N + p) * N + s) * N + r] + g2[((s * N + r) * N + q) * N + p]);
        o2[u] = 0.25 * v * inv;
    }
}

// dE/dh = gamma; dE/dg = 1/2 Gamma averaged over the 8-fold permutation
// group of (pq|rs) (the derivative along 8-fold symmetric perturbations);
// F_pq = sum_r h_pr gamma_qr + sum_rst (pr|st) Gamma_qrst, one block per
// (p, q) with a fixed-order block sum; dE/dkappa = 2 (F - F^T) in a second pass.
__global__ void k_grad_dg(int N, const double *G2, double *dg) {
    const int N2 = N * N;
    const long long N4 = (long long)N2 * N2;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < N4; u += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(u % N), r = (int)((u / N) % N), q = (int)((u / N2) % N), p = (int)(u / ((long long)N2 * N));
        auto at = [&](int a, int b, int c, int d) { return G2[((a * N + b) * N + c) * N + d]; };
        const double v = ((at(p, q, r, s) + at(q, p, r, s)) + (at(p, q, s, r) + at(q, p, s, r))) +
                         ((at(r, s, p, q) + at(s, r, p, q)) + (at(r, s, q, p) + at(s, r, q, p)));
        dg[u] = 0.0625 * v;
    }
}

__global__ void __launch_bounds__(256) k_grad_F(int N, const double *h, const double *g, const double *G1,
                                                const double *G2, double *F) {
    __shared__ double red[256];
    const int p = blockIdx.x / N, q = blockIdx.x - (blockIdx.x / N) * N;
    const int N3 = N * N * N;
    double acc = 0.0;
    for (int t = threadIdx.x; t < N3; t += blockDim.x) acc = fma(g[(size_t)p * N3 + t], G2[(size_t)q * N3 + t], acc);
    if (threadIdx.x < N) acc = fma(h[p * N + threadIdx.x], G1[q * N + threadIdx.x], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) F[blockIdx.x] = red[0];
}

__global__ void k_grad_kappa(int N, const double *F, double *dk) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * N; t += gridDim.x * blockDim.x) {
        const int p = t / N, q = t - p * N;
        dk[t] = 2.0 * (F[p * N + q] - F[q * N + p]);
    }
}

}  // namespace

cudaError_t launch_rdm(const Problem &P, IterState *st, double *g1_raw, double *g2_raw, double *norm, double *g1,
                       double *g2, cudaStream_t s) {
    const int N = P.N;
    const size_t n2 = (size_t)N * N, n4 = n2 * n2;
    cudaError_t e = cudaMemsetAsync(g1_raw, 0, n2 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g2_raw, 0, n4 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(norm, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    const size_t sh = (size_t)(N + 2 * N * N) * sizeof(double);    // up to 63 KB at N = 63
    e = cudaFuncSetAttribute(k_rdm_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
    long long blocks = (P.capacity + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_rdm_accumulate<<<(unsigned)blocks, 256, sh, s>>>(P, st, g1_raw, g2_raw, norm);
    k_rdm_finalize<<<152 * 4, 256, 0, s>>>(N, g1_raw, g2_raw, norm, g1, g2);
    return cudaGetLastError();
}

cudaError_t launch_gradient(int N, const double *h, const double *g, const double *G1, const double *G2, double *F,
                            double *dh, double *dg, double *dk, cudaStream_t s) {
    const size_t n2 = (size_t)N * N;
    cudaError_t e = cudaSuccess;
    if (dh) e = cudaMemcpyAsync(dh, G1, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    if (dg) k_grad_dg<<<152 * 4, 256, 0, s>>>(N, G2, dg);
    if (dk) {
        k_grad_F<<<N * N, 256, 0, s>>>(N, h, g, G1, G2, F);
        k_grad_kappa<<<1, 256, 0, s>>>(N, F, dk);
    }
    return cudaGetLastError();
}

}  // namespace cdfci
