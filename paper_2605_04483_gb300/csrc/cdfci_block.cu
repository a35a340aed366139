// mCDFCI (Algorithm 2): m coordinates per iteration.
//
// One iteration is a fixed sequence of kernels (captured once in a CUDA graph):
//   k_mc_gkeys     |g_j| ~ |b_j + mu c_j| of every candidate (the union of the
//                  last columns, deduplicated by a mark bit), clearing the marks;
//   k_mc_hist/scan radix selection of the m largest |g| on the 64-bit pattern,
//                  16 bits per pass;
//   k_mc_collect   the candidates above the threshold digit prefix, and the ones
//                  on it (sorted by (|g| desc, key asc) in k_mc_sortsel);
//   k_mc_prepare   c_I, b_I, H_II (Slater-Condon between the selected
//                  determinants) and H_II c_I;
//   k_mc_eigen     the reduced (m+1)-dimensional problem R = Q^T H Q with
//                  Q = [c~ / nu, E_I]; its lowest eigenpair (LOBPCG with a
//                  float-float residual, one thread per row) gives
//                  z = [nu gamma; c_I gamma + eta]; the scalars mu, alpha
//                  (double-double) and the global scale;
//   k_mc_scatter   b_j += H_ji eta_i for the m columns (compression, atomics,
//                  16-byte CAS inserts), the gather sum_j H_ji c_j per column,
//                  new candidates;
//   k_mc_finalize  the recalculated b_I, counters, snapshot.
// Stored values are c_j / s and b_j / s for a global scale s, so that
// c <- gamma c costs O(1): s <- gamma s.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "cdfci_internal.cuh"
#include "cdfci_kernels.h"

namespace cdfci {

namespace cg = cooperative_groups;

namespace {

constexpr int kInBin = 1024;          // candidates sorted in one CTA on the threshold digit

// <D1|H|D2> for two determinants differing by at most a double excitation
// (Eq. entry; same sign convention as the column enumeration: D1 is reached
// from D2 by i->a then j->b with i < j occupied, a < b empty).  Diagonal: 0
// (computed separately).
__device__ double hij_pair(const Problem &P, unsigned long long A1, unsigned long long B1, unsigned long long A2,
                           unsigned long long B2) {
    const unsigned long long dA = A1 ^ A2, dB = B1 ^ B2;
    const int la = __popcll(dA), lb = __popcll(dB);
    if (la + lb == 0 || la + lb > 4) return 0.0;
    const int N = P.N;
    const double *g = P.g;
    if (la + lb == 2) {                                  // single
        const bool alpha = la == 2;
        const unsigned long long X2 = alpha ? A2 : B2, X1 = alpha ? A1 : B1;
        const int i = __ffsll((long long)(X2 & (alpha ? dA : dB))) - 1;
        const int a = __ffsll((long long)(X1 & (alpha ? dA : dB))) - 1;
        // h_ia, then the occupied spin-orbitals of the column determinant in
        // spin-orbital order (alpha, then beta), one running sum (element_value's order); the
        // terms (ia|kk) - (ik|ka) (same spin as the excitation) and (ia|kk) come from the
        // single-excitation tables W3 and V3, eight loads in flight before their adds
        const double *rw = P.W3 + ((size_t)i * N + a) * N, *rv = P.V3 + ((size_t)i * N + a) * N;
        const double *tA = alpha ? rw : rv, *tB = alpha ? rv : rw;
        double v = __ldg(P.h + i * N + a);
        unsigned long long mA = A2, mB = B2;
        while (mA | mB) {
            double t[8];
            bool ok[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool fa = mA != 0ull;
                const unsigned long long mm = fa ? mA : mB;
                ok[u] = mm != 0ull;
                const int k = ok[u] ? __ffsll((long long)mm) - 1 : 0;
                t[u] = ok[u] ? __ldg((fa ? tA : tB) + k) : 0.0;
                if (fa) mA &= mA - 1; else mB &= mB - 1;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (ok[u]) v += t[u];
        }
        return apply_parity(v, X2 & between_mask(i, a));
    }
    if (la == 4 || lb == 4) {                            // same-spin double
        const bool alpha = la == 4;
        const unsigned long long X2 = alpha ? A2 : B2, X1 = alpha ? A1 : B1, d = alpha ? dA : dB;
        unsigned long long occ = X2 & d, vir = X1 & d;
        const int i = __ffsll((long long)occ) - 1;
        occ &= occ - 1;
        const int j = __ffsll((long long)occ) - 1;
        const int a = __ffsll((long long)vir) - 1;
        vir &= vir - 1;
        const int b = __ffsll((long long)vir) - 1;
        const unsigned long long m1 = X2 & between_mask(i, a);
        const unsigned long long Xm = X2 ^ (1ull << i) ^ (1ull << a);
        const unsigned long long m2 = Xm & between_mask(j, b);
        return apply_parity(gi(g, N, i, a, j, b) - gi(g, N, i, b, j, a), m1 ^ m2);
    }
    // opposite-spin double
    const int i = __ffsll((long long)(A2 & dA)) - 1, a = __ffsll((long long)(A1 & dA)) - 1;
    const int j = __ffsll((long long)(B2 & dB)) - 1, b = __ffsll((long long)(B1 & dB)) - 1;
    return apply_parity(gi(g, N, i, a, j, b), (A2 & between_mask(i, a)) ^ (B2 & between_mask(j, b)));
}

// ---------------------------------------------------------------------------
// Float-float numbers on the FP32 pipe (this part runs FP64 at a small
// fraction of its FP32 rate).  A value is hi + lo with |lo| <= ulp(hi) / 2,
// about 48 significant bits.  TwoSum (Knuth) and the FMA form of TwoProduct
// are error-free transformations; the _rn intrinsics keep the compiler from
// contracting or reassociating them.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// |hi| >= |lo| (or hi = 0)
__device__ __forceinline__ ff ff_norm(float hi, float lo) {
    const float s = __fadd_rn(hi, lo);
    return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    const float p = __fmul_rn(a.hi, b);
    return ff_norm(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_norm(p, e);
}
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff r = ff_add(a, ff_neg(ff_mul_f(b, q1)));
    return ff_norm(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ ff ff_from_double(double v) {
    const float hi = __double2float_rn(v);
    return {hi, __double2float_rn(v - (double)hi)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ float ff_to_float(ff a) { return __fadd_rn(a.hi, a.lo); }
// (sh, sl) += (ah + al) * x, an unnormalised float-float accumulator
__device__ __forceinline__ void ff_mac(float &sh, float &sl, float ah, float al, ff x) {
    const float p = __fmul_rn(ah, x.hi);
    float e = __fmaf_rn(ah, x.hi, -p);
    e = __fmaf_rn(ah, x.lo, e);
    e = __fmaf_rn(al, x.hi, e);
    const ff s = ff_two_sum(sh, p);
    sh = s.hi;
    sl = __fadd_rn(sl, __fadd_rn(s.lo, e));
}

// Block or cluster sums of K values held by the row leads (the other threads
// hold zero): every warp reduces in a fixed tree, lane 0 of every warp writes
// its K partials into slot (rank * warps + warp) of the scratch of every CTA
// of the cluster (CL; else its own block's), one barrier, and every thread
// adds the slots in a fixed xor butterfly, so all threads of all CTAs hold
// bit-identical sums.  Two scratch halves alternate: a half is rewritten only
// after the barrier of the following sum, which every reader of it has passed.
// The trees have a fixed depth, fully unrolled, so that the K sums interleave.
template <bool CL, int K>
__device__ __forceinline__ void bsum_f(float (&v)[K], float *scr, int &half, unsigned rank, unsigned C) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] = __fadd_rn(v[k], __shfl_down_sync(0xffffffffu, v[k], off));
    float *s = scr + half * 32 * 16;                     // fixed stride: K <= 16, slots <= 32
    const int slot = (int)rank * nw + warp, ns = (int)C * nw;
    if (lane == 0) {
        if (CL) {
            cg::cluster_group cl = cg::this_cluster();
            for (unsigned r = 0; r < C; ++r) {
                float *d = cl.map_shared_rank(s, r);
#pragma unroll
                for (int k = 0; k < K; ++k) d[slot * K + k] = v[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) s[slot * K + k] = v[k];
        }
    }
    if (CL) cg::this_cluster().sync(); else __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float t = lane < ns ? s[lane * K + k] : 0.0f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t = __fadd_rn(t, __shfl_xor_sync(0xffffffffu, t, off));
        v[k] = t;
    }
    half ^= 1;
}

template <bool CL, int K>
__device__ __forceinline__ void bsum_ff(ff (&v)[K], ff *scr, int &half, unsigned rank, unsigned C) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const ff o = {__shfl_down_sync(0xffffffffu, v[k].hi, off), __shfl_down_sync(0xffffffffu, v[k].lo, off)};
            v[k] = ff_add(v[k], o);
        }
    ff *s = scr + half * 32 * 2;                         // fixed stride: K <= 2, slots <= 32
    const int slot = (int)rank * nw + warp, ns = (int)C * nw;
    if (lane == 0) {
        if (CL) {
            cg::cluster_group cl = cg::this_cluster();
            for (unsigned r = 0; r < C; ++r) {
                ff *d = cl.map_shared_rank(s, r);
#pragma unroll
                for (int k = 0; k < K; ++k) d[slot * K + k] = v[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) s[slot * K + k] = v[k];
        }
    }
    if (CL) cg::this_cluster().sync(); else __syncthreads();
    // xor butterfly over the slots (ff_add is commutative bit for bit: TwoSum's error term is exact)
#pragma unroll
    for (int k = 0; k < K; ++k) {
        ff t = lane < ns ? s[lane * K + k] : ff{0.0f, 0.0f};
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            t = ff_add(t, ff{__shfl_xor_sync(0xffffffffu, t.hi, off), __shfl_xor_sync(0xffffffffu, t.lo, off)});
        v[k] = t;
    }
    half ^= 1;
}

// an FP64 sum over the cluster (or block) of one value per thread, in every thread (fixed order)
template <bool CL>
__device__ __forceinline__ double csum_d(double v, double *scr, unsigned rank, unsigned C) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int slot = (int)rank * nw + warp, ns = (int)C * nw;
    if (lane == 0) {
        if (CL) {
            cg::cluster_group cl = cg::this_cluster();
            for (unsigned r = 0; r < C; ++r) cl.map_shared_rank(scr, r)[slot] = v;
        } else {
            scr[slot] = v;
        }
    }
    if (CL) cg::this_cluster().sync(); else __syncthreads();
    double t = lane < ns ? scr[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    return t;
}


// Lowest eigenpair of the symmetric 3 x 3 matrix [a00 a01 a02; . a11 a12; . . a22]
// in FP32: the trigonometric form of the three real roots of the characteristic
// cubic, and the eigenvector as the longest cross product of two rows of
// (A - lambda I).  v is returned with unit length.
__device__ __forceinline__ void sym3_lowest(float a00, float a01, float a02, float a11, float a12, float a22,
                                            float &lam, float &v0, float &v1, float &v2) {
    const float sc = fmaxf(fmaxf(fmaxf(fabsf(a00), fabsf(a01)), fmaxf(fabsf(a02), fabsf(a11))),
                           fmaxf(fabsf(a12), fabsf(a22)));
    if (!(sc > 0.0f)) {
        lam = 0.0f; v0 = 1.0f; v1 = 0.0f; v2 = 0.0f;
        return;
    }
    const float is = __fdividef(1.0f, sc);
    a00 *= is; a01 *= is; a02 *= is; a11 *= is; a12 *= is; a22 *= is;
    const float q = (a00 + a11 + a22) * (1.0f / 3.0f);
    const float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    const float p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0f * (a01 * a01 + a02 * a02 + a12 * a12);
    float l = q;
    if (p2 > 0.0f) {
        const float ip = rsqrtf(p2 * (1.0f / 6.0f)), p = p2 * (1.0f / 6.0f) * ip;
        const float c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
        float r = 0.5f * (c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02));
        r = fminf(1.0f, fmaxf(-1.0f, r));
        l = q + 2.0f * p * __cosf(acosf(r) * (1.0f / 3.0f) + 2.0943951023931953f);
    }
    const float m00 = a00 - l, m11 = a11 - l, m22 = a22 - l;
    float x0 = a01 * a12 - a02 * m11, x1 = a02 * a01 - m00 * a12, x2 = m00 * m11 - a01 * a01;   // r0 x r1
    float y0 = a01 * m22 - a02 * a12, y1 = a02 * a02 - m00 * m22, y2 = m00 * a12 - a01 * a02;   // r0 x r2
    float z0 = m11 * m22 - a12 * a12, z1 = a12 * a02 - a01 * m22, z2 = a01 * a12 - m11 * a02;   // r1 x r2
    const float nx = x0 * x0 + x1 * x1 + x2 * x2, ny = y0 * y0 + y1 * y1 + y2 * y2, nz = z0 * z0 + z1 * z1 + z2 * z2;
    float n2 = nz;
    v0 = z0; v1 = z1; v2 = z2;
    if (ny > n2) { v0 = y0; v1 = y1; v2 = y2; n2 = ny; }
    if (nx > n2) { v0 = x0; v1 = x1; v2 = x2; n2 = nx; }
    if (!(n2 > 0.0f)) {              // a multiple of the identity
        v0 = 1.0f; v1 = 0.0f; v2 = 0.0f;
    } else {
        const float in = rsqrtf(n2);
        v0 *= in; v1 *= in; v2 *= in;
    }
    lam = l * sc;
}

// Lowest eigenpair of [a00 a01; a01 a11] (FP32), v of unit length.
__device__ __forceinline__ void sym2_lowest(float a00, float a01, float a11, float &lam, float &v0, float &v1) {
    const float h = 0.5f * (a00 - a11);
    const float rad = sqrtf(h * h + a01 * a01);
    lam = 0.5f * (a00 + a11) - rad;
    // (a00 - lam, a01) and (a01, a11 - lam) are rows of A - lam I; take the longer normal
    const float u0 = a01, u1 = lam - a00;             // normal of row 0
    const float w0 = a11 - lam, w1 = -a01;            // normal of row 1
    const float nu = u0 * u0 + u1 * u1, nw = w0 * w0 + w1 * w1;
    if (nu >= nw && nu > 0.0f) { const float in = rsqrtf(nu); v0 = u0 * in; v1 = u1 * in; }
    else if (nw > 0.0f) { const float in = rsqrtf(nw); v0 = w0 * in; v1 = w1 * in; }
    else { v0 = 1.0f; v1 = 0.0f; }
}
}  // namespace

// ---------------------------------------------------------------------------
// Candidates and selection (Alg. 2, choice of I): the m largest choice keys
// |b_j + mu c_j| (the bit pattern of a non-negative double orders like the
// value), ties to the smaller key.  Radix selection from the top, 12 bits per
// level (12 x 5 + 4 = 64 bits): a block counts its keys in a shared-memory
// histogram and adds it to the global one; the last block to finish (a device
// counter, after a fence) finds the digit holding the key of rank sel_need,
// narrows the prefix and clears the histogram.  Most selections resolve after
// one or two levels; later levels return at once.
// ---------------------------------------------------------------------------
constexpr int kSelBins = 4096;

// Candidates in the list: the count, clamped to the list's capacity (a count
// above it only occurs after an overflow, which set the status).
__device__ __forceinline__ int mc_ncand(const McState *ms, long long cap) {
    const long long n = ms->n_cand;
    return (int)(n < cap ? n : cap);
}
constexpr int kSelLevels = 6;

__device__ __forceinline__ int sel_bits(int level) { return level < 5 ? 12 : 4; }
__device__ __forceinline__ int sel_cover(int levels) { return levels < 6 ? 12 * levels : 64; }   // bits fixed
// the top `levels` digits of k
__device__ __forceinline__ unsigned long long sel_top(unsigned long long k, int levels) {
    const int c = sel_cover(levels);
    return c == 0 ? 0ull : (c == 64 ? k : (k >> (64 - c)));
}
__device__ __forceinline__ unsigned int sel_digit(unsigned long long k, int level) {
    const int lo = 64 - sel_cover(level + 1);
    return (unsigned int)((k >> lo) & ((1ull << sel_bits(level)) - 1ull));
}

// Add one key's digit to the block histogram sh: lanes of a warp with the same
// digit are combined first (a level's keys crowd into a few bins).  Called by
// whole warps; ok = this lane has a key to count.
__device__ __forceinline__ void sel_bin_add(unsigned int *sh, bool ok, unsigned int dg) {
    const unsigned int act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
        const unsigned int grp = __match_any_sync(act, dg);
        if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&sh[dg], (unsigned int)__popc(grp));
    }
}

// Add the block histogram to the global one (nonzero bins only); true in the
// block that finishes last.
__device__ bool sel_merge(unsigned int *sh, unsigned int *hist, unsigned int *counter) {
    __shared__ bool s_last;
    __syncthreads();
    for (int d = threadIdx.x; d < kSelBins; d += blockDim.x)
        if (sh[d]) atomicAdd(&hist[d], sh[d]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// In the last block: the digit of the key of rank need (1 = largest) among the
// counted ones; record it, clear the histogram and the counter.
__device__ void sel_scan(McState *ms, unsigned int *hist, unsigned int *counter, int level, int need) {
    __shared__ unsigned int s_warp[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int per = kSelBins / blockDim.x;             // consecutive bins per thread, from the top
    const int top = kSelBins - 1 - tid * per;
    unsigned int loc = 0;
    for (int q = 0; q < per; ++q) loc += __ldcg(&hist[top - q]);
    // exclusive prefix of loc over threads (thread 0 owns the largest digits)
    unsigned int inc = loc;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned int v = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += v;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    unsigned int base = 0;
    for (int w = 0; w < warp; ++w) base += s_warp[w];
    const unsigned int before = base + inc - loc;
    if (before < (unsigned int)need && (unsigned int)need <= before + loc) {
        unsigned int acc = before;
        for (int q = 0; q < per; ++q) {
            const unsigned int c = __ldcg(&hist[top - q]);
            if (acc + c >= (unsigned int)need) {
                ms->sel_prefix = (ms->sel_prefix << sel_bits(level)) | (unsigned long long)(top - q);
                ms->sel_need = need - (int)acc;
                ms->sel_level = level + 1;
                ms->sel_nbin = (int)c;
                ms->sel_resolved = (c <= (unsigned int)kInBin || level == kSelLevels - 1) ? 1 : 0;
                break;
            }
            acc += c;
        }
    }
    (void)nw;
    __syncthreads();
    for (int q = 0; q < per; ++q) hist[top - q] = 0u;
    if (tid == 0) *counter = 0u;
}

// choice keys of the candidates, clearing their marks; level-0 histogram
__global__ void __launch_bounds__(256) k_mc_gkeys(Problem P, McState *ms, IterState *st, const long long *cand,
                                                  unsigned long long *gkey, unsigned int *hist, int m) {
    __shared__ unsigned int sh[kSelBins];
    if (ms->done) return;
    const int n = mc_ncand(ms, P.cap_cand);
    const double mu = ms->mu.hi;
    const bool count = n > m;
    for (int d = threadIdx.x; d < kSelBins; d += blockDim.x) sh[d] = 0u;
    __syncthreads();
    const int stride = gridDim.x * blockDim.x;
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    // kGkU candidates per thread and round, all their slot loads in flight together
    constexpr int kGkU = 4;
    for (int base = blockIdx.x * blockDim.x; base < n; base += kGkU * stride) {
        long long slot[kGkU];
        bool ok[kGkU];
        double2 v[kGkU];
#pragma unroll
        for (int u = 0; u < kGkU; ++u) {
            const int t = base + u * stride + threadIdx.x;
            ok[u] = t < n;
            slot[u] = ok[u] ? cand[t] : 0;
        }
#pragma unroll
        for (int u = 0; u < kGkU; ++u) {
            v[u] = make_double2(0.0, 0.0);
            if (ok[u] && (unsigned long long)slot[u] < (unsigned long long)P.capacity)
                asm volatile("ld.global.cg.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"   // c and b of a random
                             : "=d"(v[u].x), "=d"(v[u].y)                                   // slot: evict first
                             : "l"(&P.table[slot[u]].c), "l"(pol));
        }
#pragma unroll
        for (int u = 0; u < kGkU; ++u) {
            const int t = base + u * stride + threadIdx.x;
            unsigned long long k = 0ull;
            if (ok[u] && (unsigned long long)slot[u] >= (unsigned long long)P.capacity) {
                set_status(st, kErrInternal);              // a candidate outside the table: skip it
                gkey[t] = 0ull;
            } else if (ok[u]) {
                k = (unsigned long long)__double_as_longlong(fma(mu, v[u].x, v[u].y)) & 0x7fffffffffffffffull;
                gkey[t] = k;
                mark_clear(P, slot[u]);                    // clear the candidate mark
            }
            if (count) sel_bin_add(sh, ok[u], sel_digit(k, 0));
        }
    }
    if (!count) {                                      // every candidate is chosen
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ms->sel_prefix = 0ull;
            ms->sel_need = 0;
            ms->sel_level = 0;
            ms->sel_nbin = 0;
            ms->sel_resolved = 1;
        }
        return;
    }
    if (sel_merge(sh, hist, hist + kSelBins)) {
        if (threadIdx.x == 0) ms->sel_prefix = 0ull;
        __syncthreads();
        sel_scan(ms, hist, hist + kSelBins, 0, m);
    }
}

// Levels 2.. by the block that finished level 1 (1024 threads): it stops at once
// when the selection is resolved, which is the common case; otherwise it counts
// the keys on the prefix in a shared-memory histogram and scans it, level by
// level, exactly as the level-1 pass and sel_scan do.
__device__ void mc_hist_tail(McState *ms, const unsigned long long *gkey, long long cap, unsigned int *sh) {
    __shared__ unsigned int s_warp[32];
    __shared__ int s_stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int level = 2; level < kSelLevels; ++level) {
        if (tid == 0) s_stop = (ms->done || ms->sel_resolved) ? 1 : 0;
        for (int d = tid; d < kSelBins; d += blockDim.x) sh[d] = 0u;
        __syncthreads();
        if (s_stop) return;                               // uniform
        const int n = mc_ncand(ms, cap);
        const unsigned long long prefix = ms->sel_prefix;
        const int need = ms->sel_need;
        for (int base = 0; base < n; base += blockDim.x) {
            const int t = base + tid;
            const unsigned long long k = t < n ? gkey[t] : 0ull;
            const bool ok = t < n && sel_top(k, level) == prefix;
            sel_bin_add(sh, ok, sel_digit(k, level));
        }
        __syncthreads();
        // the digit of rank `need` from the top (thread t owns bins top - t per .. top - t per - per + 1)
        const int per = kSelBins / blockDim.x;
        const int top = kSelBins - 1 - tid * per;
        unsigned int loc = 0;
        for (int q = 0; q < per; ++q) loc += sh[top - q];
        unsigned int inc = loc;
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned int v = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += v;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        unsigned int before = inc - loc;
        for (int w2 = 0; w2 < warp; ++w2) before += s_warp[w2];
        if (before < (unsigned int)need && (unsigned int)need <= before + loc) {
            unsigned int acc = before;
            for (int q = 0; q < per; ++q) {
                const unsigned int c = sh[top - q];
                if (acc + c >= (unsigned int)need) {
                    ms->sel_prefix = (ms->sel_prefix << sel_bits(level)) | (unsigned long long)(top - q);
                    ms->sel_need = need - (int)acc;
                    ms->sel_level = level + 1;
                    ms->sel_nbin = (int)c;
                    ms->sel_resolved = (c <= (unsigned int)kInBin || level == kSelLevels - 1) ? 1 : 0;
                    break;
                }
                acc += c;
            }
        }
        __threadfence_block();
        __syncthreads();
    }
}

// level 1 on the grid: the keys on the level-0 prefix; the last block to merge
// its histogram scans it and goes on with the levels below (mc_hist_tail)
constexpr int kHistThreads = 1024;
__global__ void __launch_bounds__(kHistThreads) k_mc_hist(McState *ms, const unsigned long long *gkey,
                                                          unsigned int *hist, long long cap) {
    __shared__ unsigned int sh[kSelBins];
    const int level = 1;
    if (ms->done || ms->sel_resolved) return;
    const int n = mc_ncand(ms, cap);
    const unsigned long long prefix = ms->sel_prefix;
    const int need = ms->sel_need;
    for (int d = threadIdx.x; d < kSelBins; d += blockDim.x) sh[d] = 0u;
    __syncthreads();
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int t = base + threadIdx.x;
        unsigned long long k = t < n ? gkey[t] : 0ull;
        const bool ok = t < n && sel_top(k, level) == prefix;
        sel_bin_add(sh, ok, sel_digit(k, level));
    }
    if (sel_merge(sh, hist, hist + kSelBins)) {
        sel_scan(ms, hist, hist + kSelBins, level, need);
        __threadfence_block();
        __syncthreads();                                // the scan's McState fields visible to the block
        mc_hist_tail(ms, gkey, cap, sh);
    }
}

__global__ void k_mc_collect(Problem P, McState *ms, const long long *cand, const unsigned long long *gkey,
                             McSel *sel, McSel *inbin) {
    if (ms->done) return;
    const int n = mc_ncand(ms, P.cap_cand);
    const bool all = ms->sel_level == 0;                 // n_cand <= m: every candidate is selected
    const int L = ms->sel_level;
    const unsigned long long prefix = ms->sel_prefix;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const unsigned long long k = gkey[t];
        const unsigned long long top = sel_top(k, L);
        McSel x;
        x.slot = cand[t];
        x.gkey = k;
        if (all || top > prefix) {
            const int pos = atomicAdd(&ms->n_above, 1);
            const Slot s = P.table[x.slot];
            x.A = s.a;
            x.B = s.b & kKeyMaskB;
            sel[pos] = x;
        } else if (top == prefix) {
            const int pos = atomicAdd(&ms->n_inbin, 1);
            if (pos < kInBin) {
                const Slot s = P.table[x.slot];
                x.A = s.a;
                x.B = s.b & kKeyMaskB;
                inbin[pos] = x;
            }
        }
    }
}

// Exact ties beyond the in-bin capacity: when every 64 bits of the choice key
// are fixed and more than kInBin candidates carry that key, the sel_need
// smallest determinant keys among them are chosen (ties go to the smaller key)
// by a radix selection on the 128-bit key (B, A), 8 bits per pass from the
// top, in one CTA over a compacted copy of the tied candidates.  The chosen
// ones replace the in-bin buffer.  Symmetric lattices produce such groups.
// Run by the sorting CTA before it sorts (the caller has checked the
// condition; block-uniform).
__device__ void mc_ties(const Problem &P, McState *ms, const long long *cand, const unsigned long long *gkey,
                        McSel *ties, McSel *inbin) {
    __shared__ unsigned int hist[256];
    __shared__ int s_n, s_out, s_digit;
    __shared__ unsigned int s_below;
    const int n = mc_ncand(ms, P.cap_cand), tid = threadIdx.x;
    const unsigned long long g = ms->sel_prefix;
    int need = ms->sel_need;
    if (tid == 0) { s_n = 0; s_out = 0; }
    __syncthreads();
    for (int t = tid; t < n; t += blockDim.x) {
        if (gkey[t] != g) continue;
        const Slot sl = P.table[cand[t]];
        ties[atomicAdd(&s_n, 1)] = McSel{cand[t], g, sl.a, sl.b & kKeyMaskB};
    }
    __syncthreads();
    const int nt = s_n;
    // digit q of the key: bits [120 - 8q, 128 - 8q) of (B << 64) | A
    unsigned long long pB = 0ull, pA = 0ull;           // the fixed top digits (as bit patterns)
    int fixed = 0;                                     // bits fixed so far
    for (int q = 0; q < 16 && need > 0; ++q) {
        for (int d = tid; d < 256; d += blockDim.x) hist[d] = 0u;
        __syncthreads();
        for (int t = tid; t < nt; t += blockDim.x) {
            const McSel x = ties[t];
            const bool on = fixed == 0 ||
                            (fixed <= 64 ? (x.B >> (64 - fixed)) == (pB >> (64 - fixed))
                                         : (x.B == pB && (x.A >> (128 - fixed)) == (pA >> (128 - fixed))));
            if (!on) continue;
            const unsigned int dg = q < 8 ? (unsigned int)((x.B >> (56 - 8 * q)) & 0xffu)
                                          : (unsigned int)((x.A >> (56 - 8 * (q - 8))) & 0xffu);
            atomicAdd(&hist[dg], 1u);
        }
        __syncthreads();
        if (tid == 0) {
            unsigned int acc = 0;
            int d = 0;
            for (; d < 256; ++d) {
                if (acc + hist[d] >= (unsigned int)need) break;
                acc += hist[d];
            }
            s_digit = d;
            s_below = acc;
        }
        __syncthreads();
        const int dsel = s_digit;
        // every key on the prefix with a smaller digit is chosen
        for (int t = tid; t < nt; t += blockDim.x) {
            const McSel x = ties[t];
            const bool on = fixed == 0 ||
                            (fixed <= 64 ? (x.B >> (64 - fixed)) == (pB >> (64 - fixed))
                                         : (x.B == pB && (x.A >> (128 - fixed)) == (pA >> (128 - fixed))));
            if (!on) continue;
            const int dg = q < 8 ? (int)((x.B >> (56 - 8 * q)) & 0xffu) : (int)((x.A >> (56 - 8 * (q - 8))) & 0xffu);
            if (dg < dsel) inbin[atomicAdd(&s_out, 1)] = x;
        }
        need -= (int)s_below;
        if (q < 8) pB |= (unsigned long long)dsel << (56 - 8 * q);
        else pA |= (unsigned long long)dsel << (56 - 8 * (q - 8));
        fixed += 8;
        __syncthreads();
    }
    // keys are unique, so after the last digit exactly `need` (0 or 1) entries match the full key
    if (need > 0)
        for (int t = tid; t < nt; t += blockDim.x) {
            const McSel x = ties[t];
            if (x.B == pB && x.A == pA) inbin[atomicAdd(&s_out, 1)] = x;
        }
    __syncthreads();
    if (tid == 0) ms->n_inbin = s_out;                 // = sel_need
    __threadfence_block();
    __syncthreads();
}

// Bitonic sort, in shared memory, of (choice key, index) pairs into the choice
// order: |g| descending, then the determinant key ascending (looked up in src
// for exact ties only).  Padding entries (index -1) sort last.
// One element of a sort, held in registers: the choice key and the determinant
// (a strict total order: keys are unique); padding sorts last.
struct SelE {
    unsigned long long g, A, B;
    long long slot;
};
__device__ __forceinline__ bool sel_first(const SelE &x, const SelE &y) {   // x before y in the choice order
    if (x.g != y.g) return x.g > y.g;
    return key_less(x.A, x.B, y.A, y.B);
}
__device__ __forceinline__ SelE sel_pad() { return SelE{0ull, ~0ull, ~0ull, -1}; }
// Bitonic sort into the choice order of n_pow2 elements, one per thread (thread
// t holds element t; n_pow2 a power of two).  Only the first max(n_pow2, 32)
// threads take part (the caller's other threads skip it): a stage whose
// partners lie in one warp (distance < 32) exchanges by shuffles, the others
// through buf between two barriers of the taking-part warps (named barrier 1).
__device__ void bitonic_reg(SelE &e, int n_pow2, SelE *buf) {
    const int t = threadIdx.x;
    const int nact = n_pow2 < 32 ? 32 : n_pow2;
    for (int k = 2; k <= n_pow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            SelE o;
            if (j >= 32) {                              // uniform
                buf[t] = e;
                asm volatile("bar.sync 1, %0;" ::"r"(nact) : "memory");
                o = buf[t ^ j];
                asm volatile("bar.sync 1, %0;" ::"r"(nact) : "memory");
            } else {
                o.g = __shfl_xor_sync(0xffffffffu, e.g, j);
                o.A = __shfl_xor_sync(0xffffffffu, e.A, j);
                o.B = __shfl_xor_sync(0xffffffffu, e.B, j);
                o.slot = __shfl_xor_sync(0xffffffffu, e.slot, j);
            }
            // the lower position of an ascending pair (and the upper of a descending one) keeps the
            // first of the two
            const bool keep_first = ((t & j) == 0) == ((t & k) == 0);
            const bool o_first = sel_first(o, e), e_first = sel_first(e, o);
            if (keep_first ? o_first : e_first) e = o;
        }
    }
}

// The in-bin candidates sorted (after the exact-tie pass when more than kInBin
// share the whole 64-bit choice key), the first sel_need of them join the
// chosen set; then the chosen set in the choice order (a canonical order for
// the reduced problem's rows).  1024 threads, one element each.
__global__ void __launch_bounds__(1024) k_mc_sortsel(Problem P, McState *ms, McSel *sel, McSel *inbin, int m,
                                                      IterState *st, const long long *cand,
                                                      const unsigned long long *gkey, McSel *ties) {
    __shared__ SelE buf[kInBin];
    const int tid = threadIdx.x;
    if (ms->done) return;
    if (ms->sel_level >= kSelLevels && ms->n_inbin > kInBin) mc_ties(P, ms, cand, gkey, ties, inbin);   // uniform
    const int n_above = ms->n_above;
    int n_in = ms->n_inbin;
    if (ms->sel_level > 0 && n_in > kInBin) {
        if (tid == 0) set_status(st, kErrArg);            // more than kInBin candidates with one key pattern
        n_in = kInBin;
    }
    const int need = ms->sel_level == 0 ? 0 : ms->sel_need;
    const int take = need < n_in ? need : n_in;
    if (take > 0) {                                     // uniform
        int p2 = 1;
        while (p2 < n_in) p2 <<= 1;
        SelE e = sel_pad();
        if (tid < n_in) { const McSel x = inbin[tid]; e = SelE{x.gkey, x.A, x.B, x.slot}; }
        if (n_in > 1 && tid < (p2 < 32 ? 32 : p2)) bitonic_reg(e, p2, buf);
        if (tid < take) sel[n_above + tid] = McSel{e.slot, e.g, e.A, e.B};
        __syncthreads();                                // sel visible to the block
    }
    const int msel = n_above + take;
    if (msel > 1) {
        int q2 = 1;
        while (q2 < msel) q2 <<= 1;
        SelE e = sel_pad();
        if (tid < msel) { const McSel x = sel[tid]; e = SelE{x.gkey, x.A, x.B, x.slot}; }
        if (tid < (q2 < 32 ? 32 : q2)) bitonic_reg(e, q2, buf);
        if (tid < msel) sel[tid] = McSel{e.slot, e.g, e.A, e.B};
    }
    if (tid == 0) {
        ms->m_sel = msel;
        ms->n_above = 0;
        ms->n_inbin = 0;
    }
}

constexpr int kEigMaxN = 1024;      // m + 1 <= 1024: one thread per row of the reduced problem

// The entries of the column of {A, B} into tab, threads t0, t0 + nt, ...
__device__ __forceinline__ void mc_build_coltab(const Problem &P, const ColLists &L, unsigned long long A,
                                                unsigned long long B, ColEnt *tab, int t0, int nt) {
    const int na_va = P.na * P.va, nb_vb = P.nb * P.vb, N = P.N;
    for (int s = t0; s < na_va + nb_vb; s += nt) {
        const bool alpha = s < na_va;
        const int sl = alpha ? s : s - na_va;
        const int o = (int)fdiv((unsigned)sl, alpha ? P.mg_va : P.mg_vb);
        const int w = sl - o * (alpha ? P.va : P.vb);
        const int i = alpha ? L.occA[o] : L.occB[o];
        const int a = alpha ? L.virA[w] : L.virB[w];
        const unsigned long long X = alpha ? A : B;
        ColEnt e;
        e.key = X ^ (1ull << i) ^ (1ull << a);
        e.h = alpha ? hash_alpha(e.key) : hash_beta(e.key);
        e.goff = alpha ? (i * N + a) * N * N : i * N + a;
        e.info = (__popcll(X & between_mask(i, a)) & 1) | (i << 8) | (a << 16) |
                 (P.ksub ? (int)__ldg(P.ksub + i * N + a) << 24 : 0);
        e.pad0 = 0;
        e.pad1 = 0;
        tab[s] = e;
    }
}

// ---------------------------------------------------------------------------
// c_I, b_I, H_II, H_II c_I: one warp per selected row.  H_II goes to rows and
// columns 1..m of R as float-float pairs (Rh, Rl; leading dimension ldr).
// ---------------------------------------------------------------------------
constexpr int kPrepWarps = 8;       // rows (warps) per block

__global__ void __launch_bounds__(32 * kPrepWarps) k_mc_prepare(Problem P, McState *ms, const McSel *sel, double *cI,
                                                    double *bI, double *Hdiag, double *HIIc, float4 *rowf, float *Rh,
                                                    float *Rl, int ldr, ColEnt *coltab, ColLists *collists, int ns) {
    __shared__ ColLists Lw[kPrepWarps];
    // the chosen determinants and their c (true units), staged once per block
    __shared__ unsigned long long s_A[kEigMaxN], s_B[kEigMaxN];
    __shared__ double s_c[kEigMaxN];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (ms->done) return;
    const int m = ms->m_sel;
    const double s = ms->scale.hi;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const McSel x = sel[i];
        s_A[i] = x.A;
        s_B[i] = x.B;
        s_c[i] = P.table[x.slot].c * s;
    }
    __syncthreads();
    for (int r = blockIdx.x * kPrepWarps + warp; r < m; r += gridDim.x * kPrepWarps) {
        const unsigned long long rA = s_A[r], rB = s_B[r];
        const double b_r = lane == 0 ? P.table[sel[r].slot].bv : 0.0;     // issued early: a random slot
        ColLists &L = Lw[warp];
        for (int t = lane; t < P.N; t += 32) {
            int ra = __popcll(rA & low_mask(t)), rb = __popcll(rB & low_mask(t));
            if ((rA >> t) & 1ull) L.occA[ra] = (unsigned char)t; else L.virA[t - ra] = (unsigned char)t;
            if ((rB >> t) & 1ull) L.occB[rb] = (unsigned char)t; else L.virB[t - rb] = (unsigned char)t;
        }
        __syncwarp();
        // the column's single excitations and orbital lists for the scatter
        mc_build_coltab(P, L, rA, rB, coltab + (size_t)r * ns, lane, 32);
        reinterpret_cast<uint2 *>(collists + r)[lane] = reinterpret_cast<const uint2 *>(&L)[lane];
        const double hd = diag_warp(P, L);
        // (pairs more than a double excitation apart, or doubles when every double vanishes, are zero:
        // no FP64 work for them; a zero term leaves acc unchanged)
        const int dmax = P.doubles_vanish ? 2 : 4;
        double acc = 0.0;
        for (int c = lane; c < m; c += 32) {
            const unsigned long long cA = s_A[c], cB = s_B[c];
            const int dd2 = __popcll(rA ^ cA) + __popcll(rB ^ cB);
            float hh = 0.0f, hl = 0.0f;
            if (c == r || (dd2 > 0 && dd2 <= dmax)) {
                const double h = (c == r) ? hd : hij_pair(P, rA, rB, cA, cB);
                const ff hf = ff_from_double(h);
                hh = hf.hi;
                hl = hf.lo;
                acc = fma(h, s_c[c], acc);
            }
            Rh[(size_t)(r + 1) * ldr + (c + 1)] = hh;
            Rl[(size_t)(r + 1) * ldr + (c + 1)] = hl;
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        // the row's values, and for the reduced solve c_r, b_r, (H_II c_I)_r, b_r - (H_II c_I)_r as
        // float-float pairs (lanes 0..3, one conversion each)
        const double hc = __shfl_sync(0xffffffffu, acc, 0), br = __shfl_sync(0xffffffffu, b_r, 0) * s;
        if (lane == 0) {
            cI[r] = s_c[r];
            bI[r] = br;
            Hdiag[r] = hd;
            HIIc[r] = hc;
        }
        const double cv = lane == 0 ? s_c[r] : (lane == 1 ? br : (lane == 2 ? hc : br - hc));
        const ff f = ff_from_double(cv);
        const float fh1 = __shfl_sync(0xffffffffu, f.hi, lane | 1), fl1 = __shfl_sync(0xffffffffu, f.lo, lane | 1);
        if (lane == 0 || lane == 2) rowf[2 * r + (lane >> 1)] = make_float4(f.hi, f.lo, fh1, fl1);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// The reduced problem: the lowest eigenpair of the active block A of
// R = Q^T H Q, Q = [c~ / nu, E_I] (rows/columns 1.. only when c lies in
// span(E_I)), on one CTA with one thread group per row.
//
// LOBPCG (Knyazev's locally optimal block preconditioned conjugate gradient)
// for one vector, with the diagonal (Davidson) preconditioner, started from
// the current point x = [nu; c_I], whose image is known without a product:
// (A x)_i = nu R_i0 + (H_II c_I)_i = b_i and (A x)_0 = (alpha - c_I.b_I) / nu.
// x and A x are float-float; the search vectors w, p and their images are
// FP32.  The Rayleigh-Ritz step on span{x, w, p} uses the float-float residual
// r = A x - theta x for the x-couplings (x^T A w = r^T w once w is orthogonal
// to x), so the iteration converges to the accuracy of the float-float
// residual, about 1e-14 relative, with all vector arithmetic on the FP32 pipe.
// FP64 is kept to the few scalars that need its range or its cancellation-free
// sums; on this part a dependent FP64 operation costs far more than an FP32 one.
//
// Vectors are held in the absolute indexing of R (entry 0 is the direction
// c~ / nu, zero when it is not active) and padded with zeros to a multiple of
// 4 entries, so that a row of A times a vector reads 16 bytes per load along
// the row (R is symmetric).
// ---------------------------------------------------------------------------
constexpr int kEigSmemN = 160;      // A in shared memory (hi and lo) up to this size
constexpr int kEigMaxIt = 200;

// How the reduced problem of size n1 = m + 1 is laid out:
//   n1 <= kEigSmemN: one CTA, R in its shared memory, 2 threads per row;
//   else a cluster of C = 2, 4 or 8 CTAs, each holding a block of `crows` rows
//   of R (hi and lo) in its shared memory, tpr threads per row, when such a
//   split fits (at most 32 warps in the cluster, the rows within
//   kEigClusterBytes per CTA);
//   else one CTA streaming R from global memory (C = 0), 1 thread per row.
constexpr size_t kEigClusterBytes = 192 * 1024;
struct EigCfg {
    int C, tpr, crows;
};
__host__ __device__ __forceinline__ EigCfg eig_cfg(int n1) {
    if (n1 <= kEigSmemN) return EigCfg{1, 2, n1};
    for (int C = 2; C <= 8; C *= 2) {
        const int crows = (n1 + C - 1) / C;
        for (int tpr = 2; tpr >= 1; --tpr) {
            const int nw = tpr * ((crows + 31) / 32);
            const size_t ldr = 32 * (size_t)((n1 + 31) / 32) + 4 * (size_t)tpr;
            if (C * nw <= 32 && 8 * (size_t)crows * ldr <= kEigClusterBytes) return EigCfg{C, tpr, crows};
        }
    }
    return EigCfg{0, 1, n1};
}
// threads per row and R's row stride: a multiple of 32 floats plus 4 tpr, which
// puts the 16-byte loads of a quarter warp (8 lanes: 8 / tpr rows, tpr chunks
// each) on distinct banks; the same stride in global and shared memory makes
// each CTA's block of rows one contiguous bulk copy
__host__ __device__ __forceinline__ int eig_tpr(int n1) { return eig_cfg(n1).tpr; }
__host__ __device__ __forceinline__ int eig_ldr(int n1) { return 32 * ((n1 + 31) / 32) + 4 * eig_tpr(n1); }
// entries of a vector in absolute indexing, a multiple of 4
__host__ __device__ __forceinline__ int eig_len(int n1) { return 4 * ((n1 + 3) / 4); }

// Row ra of R times a vector v (absolute indexing, nq chunks of 4 entries):
// this thread's share, the chunks q = k, k + tpr, ... (k = its rank in the
// row's group of tpr threads), U chunks of A in flight per round.
template <int U>
__device__ __forceinline__ float f_row_part(const float *A, int ld, int nq, int ra, int k, int tpr, const float *v) {
    const float4 *a4 = reinterpret_cast<const float4 *>(A + (size_t)ra * ld);
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
    float acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = 0.0f;
    int q = k;
    for (; q + (U - 1) * tpr < nq; q += U * tpr) {
        float4 av[U];
#pragma unroll
        for (int u = 0; u < U; ++u) av[u] = a4[q + u * tpr];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float4 x = v4[q + u * tpr];
            acc[u] = fmaf(av[u].x, x.x, acc[u]);
            acc[u] = fmaf(av[u].y, x.y, acc[u]);
            acc[u] = fmaf(av[u].z, x.z, acc[u]);
            acc[u] = fmaf(av[u].w, x.w, acc[u]);
        }
    }
    for (; q < nq; q += tpr) {
        const float4 a = a4[q], x = v4[q];
        acc[0] = fmaf(a.x, x.x, acc[0]);
        acc[0] = fmaf(a.y, x.y, acc[0]);
        acc[0] = fmaf(a.z, x.z, acc[0]);
        acc[0] = fmaf(a.w, x.w, acc[0]);
    }
    float t = acc[0];
#pragma unroll
    for (int u = 1; u < U; ++u) t += acc[u];
    return t;
}
// the same for float-float A (hi, lo) and x (pairs x[2 j], x[2 j + 1])
template <int U>
__device__ __forceinline__ ff ff_row_part(const float *Ah, const float *Al, int ld, int nq, int ra, int k, int tpr,
                                          const float *x) {
    const float4 *h4 = reinterpret_cast<const float4 *>(Ah + (size_t)ra * ld);
    const float4 *l4 = reinterpret_cast<const float4 *>(Al + (size_t)ra * ld);
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    float sh[2] = {0.0f, 0.0f}, sl[2] = {0.0f, 0.0f};
    int q = k;
    for (; q + (U - 1) * tpr < nq; q += U * tpr) {
        float4 hv[U], lv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            hv[u] = h4[q + u * tpr];
            lv[u] = l4[q + u * tpr];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = q + u * tpr, a = u & 1;
            const float4 xa = x4[2 * c], xb = x4[2 * c + 1];
            ff_mac(sh[a], sl[a], hv[u].x, lv[u].x, ff{xa.x, xa.y});
            ff_mac(sh[a], sl[a], hv[u].y, lv[u].y, ff{xa.z, xa.w});
            ff_mac(sh[a], sl[a], hv[u].z, lv[u].z, ff{xb.x, xb.y});
            ff_mac(sh[a], sl[a], hv[u].w, lv[u].w, ff{xb.z, xb.w});
        }
    }
    for (; q < nq; q += tpr) {
        const float4 h = h4[q], l = l4[q], xa = x4[2 * q], xb = x4[2 * q + 1];
        ff_mac(sh[0], sl[0], h.x, l.x, ff{xa.x, xa.y});
        ff_mac(sh[0], sl[0], h.y, l.y, ff{xa.z, xa.w});
        ff_mac(sh[0], sl[0], h.z, l.z, ff{xb.x, xb.y});
        ff_mac(sh[0], sl[0], h.w, l.w, ff{xb.z, xb.w});
    }
    return ff_add(ff_norm(sh[0], sl[0]), ff_norm(sh[1], sl[1]));
}
// sums over the tpr lanes of a row's group (xor butterfly: sums of commutative
// pairs, identical in every lane of the group)
__device__ __forceinline__ ff ff_group_sum(ff v, int tpr) {
    for (int o = 1; o < tpr; o <<= 1)
        v = ff_add(v, ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
    return v;
}
__device__ __forceinline__ float f_group_sum(float v, int tpr) {
    for (int o = 1; o < tpr; o <<= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// A x (float-float) and A w (FP32) for the row; every lane of the group holds
// it.  2 (float-float) or 4 (FP32) chunks of the row in flight per round
// (more would spill at the 64 registers of a 1024-thread block).
__device__ __forceinline__ ff ff_row(const float *Ah, const float *Al, int ld, int nq, int ra, int k, int tpr,
                                     bool act, const float *x) {
    return ff_group_sum(act ? ff_row_part<2>(Ah, Al, ld, nq, ra, k, tpr, x) : ff{0.0f, 0.0f}, tpr);
}
__device__ __forceinline__ float f_row(const float *Ah, int ld, int nq, int ra, int k, int tpr, bool act,
                                       const float *w) {
    return f_group_sum(act ? f_row_part<4>(Ah, ld, nq, ra, k, tpr, w) : 0.0f, tpr);
}

// float-float 1 / sqrt(a), a > 0 and normal in FP32: the FP32 estimate and two
// Newton steps y <- y + y (1 - a y^2) / 2 (Newton's iteration for the inverse
// square root), the residual 1 - a y^2 formed in float-float; each step about
// doubles the correct bits, up to the format's ~48.
__device__ __forceinline__ ff ff_rsqrt(ff a) {
    ff y = {rsqrtf(a.hi), 0.0f};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const ff e = ff_add(ff{1.0f, 0.0f}, ff_neg(ff_mul(a, ff_mul(y, y))));
        y = ff_add(y, ff_mul_f(y, 0.5f * e.hi));
    }
    return y;
}

// Bulk copies global -> shared by the TMA unit (cp.async.bulk), completed on an
// mbarrier by transaction bytes: one thread arms the barrier with the total,
// the lanes of one warp issue one copy per row, every thread later waits for
// the barrier's phase 0.  Addresses 16-byte aligned, sizes multiples of 16.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init_arm(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// true once the barrier's phase of the given parity has completed; gives up after `limit` polls
__device__ __forceinline__ bool mbar_wait_parity(unsigned long long *bar, unsigned parity, int limit) {
    for (int i = 0; i < limit; ++i) {
        unsigned ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}
// true once phase 0 of the barrier has completed; gives up after `limit` polls
__device__ __forceinline__ bool mbar_wait0(unsigned long long *bar, int limit) {
    for (int i = 0; i < limit; ++i) {
        unsigned ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok) : "r"(smem_u32(bar)) : "memory");
        if (ok) return true;
    }
    return false;
}

// FP64 sums over a warp of four values at once (a butterfly that halves the
// values while it halves the lanes: 6 dependent adds instead of 4 x 5); lane l
// ends with the sum of value l >> 3, in a fixed order
__device__ __forceinline__ double wsum4(double a, double b, double c, double d) {
    const int lane = threadIdx.x & 31;
    const bool up = lane & 16;
    double x0 = up ? c : a, x1 = up ? d : b;
    x0 += __shfl_xor_sync(0xffffffffu, up ? a : c, 16);
    x1 += __shfl_xor_sync(0xffffffffu, up ? b : d, 16);
    const bool up2 = lane & 8;
    double z = up2 ? x1 : x0;
    z += __shfl_xor_sync(0xffffffffu, up2 ? x0 : x1, 8);
    z += __shfl_xor_sync(0xffffffffu, z, 4);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    return z;
}

// Dynamic shared memory of k_mc_eigen, in floats: A (hi, lo) when it fits,
// then x (float-float), w, z (FP64) and a staging area, each of eig_len(m + 1)
// entries in absolute indexing.
__host__ __device__ __forceinline__ size_t eig_vec_floats(int n1) { return 7 * (size_t)eig_len(n1); }
// R in global memory: the rows per stage buffer (two buffers, each hi and lo rows x ldr floats, about
// 160 KB in all) and the product results (2 eig_len floats) after the vectors
constexpr size_t kEigStageBytes = 160 * 1024;
__host__ __device__ __forceinline__ int eig_stage_rows(int n1) {
    const int ldr = eig_ldr(n1), r = (int)(kEigStageBytes / (16 * (size_t)ldr));
    return r < 1 ? 1 : (r > n1 ? n1 : r);
}

// R in global memory: y = R v for rows 0..m, R passing through two stage
// buffers in shared memory (TMA bulk copies of contiguous row blocks, one
// mbarrier per buffer, issued by thread 0 two blocks ahead); every thread
// works on every staged block, g threads per row (a power of two), and the
// row's sum goes to y (FP32 y[r], or float-float y[2 r], y[2 r + 1]).  v is
// in absolute indexing (float-float pairs for FF), nq chunks of 4 entries.
// par[b] is the parity of buffer b's next phase; a wait that gives up sets
// the status (the copies are then waited for once more, bounded, at the end).
template <bool FF>
__device__ void eig_stream(const float *Rh, const float *Rl, int ldr, int n1, int nq, float *buf, int rows,
                           unsigned long long *bar, unsigned (&par)[2], const float *v, float *y, IterState *st) {
    const int tid = threadIdx.x, nt = blockDim.x;
    int g = 1;
    while (g < 32 && 2 * g * rows <= nt) g <<= 1;
    const int nch = (n1 + rows - 1) / rows;
    const size_t stage = 2 * (size_t)rows * ldr;      // floats per buffer (hi rows, then lo rows)
    auto issue = [&](int c) {
        const int r0 = c * rows, nr = min(rows, n1 - r0), b = c & 1;
        const unsigned bytes = (unsigned)nr * (unsigned)ldr * 4u;
        float *dst = buf + b * stage;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     ::"r"(smem_u32(bar + b)), "r"(FF ? 2u * bytes : bytes) : "memory");
        bulk_g2s(dst, Rh + (size_t)r0 * ldr, bytes, bar + b);
        if (FF) bulk_g2s(dst + (size_t)rows * ldr, Rl + (size_t)r0 * ldr, bytes, bar + b);
    };
    if (tid == 0) {
        issue(0);
        if (nch > 1) issue(1);
    }
    bool late = false;
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1, r0 = c * rows, nr = min(rows, n1 - r0);
        late |= !mbar_wait_parity(bar + b, par[b], 1 << 22);
        par[b] ^= 1u;
        const float *bh = buf + b * stage, *bl = bh + (size_t)rows * ldr;
        const int rr = tid / g, k = tid - rr * g;
        if (FF) {
            float sh0 = 0.0f, sl0 = 0.0f;
            if (rr < nr) {
                const float4 *h4 = reinterpret_cast<const float4 *>(bh + (size_t)rr * ldr);
                const float4 *l4 = reinterpret_cast<const float4 *>(bl + (size_t)rr * ldr);
                const float4 *x4 = reinterpret_cast<const float4 *>(v);
                for (int q = k; q < nq; q += g) {
                    const float4 h = h4[q], l = l4[q], xa = x4[2 * q], xb = x4[2 * q + 1];
                    ff_mac(sh0, sl0, h.x, l.x, ff{xa.x, xa.y});
                    ff_mac(sh0, sl0, h.y, l.y, ff{xa.z, xa.w});
                    ff_mac(sh0, sl0, h.z, l.z, ff{xb.x, xb.y});
                    ff_mac(sh0, sl0, h.w, l.w, ff{xb.z, xb.w});
                }
            }
            ff t = ff_norm(sh0, sl0);
            for (int o = 1; o < g; o <<= 1)
                t = ff_add(t, ff{__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)});
            if (rr < nr && k == 0) { y[2 * (r0 + rr)] = t.hi; y[2 * (r0 + rr) + 1] = t.lo; }
        } else {
            float a0 = 0.0f, a1 = 0.0f;
            if (rr < nr) {
                const float4 *h4 = reinterpret_cast<const float4 *>(bh + (size_t)rr * ldr);
                const float4 *w4 = reinterpret_cast<const float4 *>(v);
                for (int q = k; q < nq; q += g) {
                    const float4 h = h4[q], x = w4[q];
                    a0 = fmaf(h.x, x.x, a0);
                    a1 = fmaf(h.y, x.y, a1);
                    a0 = fmaf(h.z, x.z, a0);
                    a1 = fmaf(h.w, x.w, a1);
                }
            }
            float t = a0 + a1;
            for (int o = 1; o < g; o <<= 1) t = __fadd_rn(t, __shfl_xor_sync(0xffffffffu, t, o));
            if (rr < nr && k == 0) y[r0 + rr] = t;
        }
        __syncthreads();                                // buffer b read by every thread; y complete at the end
        if (tid == 0 && c + 2 < nch) issue(c + 2);
    }
    if (late) set_status(st, kErrTimeout);
}

// CL = false: one CTA holds the whole problem (R in its shared memory when
// SM, else streamed from global memory); CL = true (with SM): a cluster of C CTAs,
// CTA r holding rows [r crows, (r + 1) crows) of R in its shared memory, the
// vectors x and w gathered in full in every CTA before each product, the sums
// taken over the cluster.  Every CTA computes the scalar steps itself, from
// the same sums in the same order, so they agree bit for bit.
// (SM is a template parameter so that each instantiation holds only the code it runs: the kernel runs
// once per iteration on whichever SM is free, its instructions fetched from L2 each time.)
template <bool CL, bool SM>
__global__ void __launch_bounds__(kEigMaxN) k_mc_eigen(Problem P, McState *ms, IterState *st, const McSel *sel,
                                                       const double *cI, const double *bI, const double *HIIc,
                                                       const double *Hdiag, const float4 *rowf, float *Rh, float *Rl,
                                                       int ldr, int tpr, int crows, double *w,
                                                       double *thr, double *etaout) {
    extern __shared__ __align__(16) float sm[];
    __shared__ float s_rf[2 * 32 * 16];
    __shared__ ff s_rff[2 * 32 * 2];
    __shared__ double s_red[32 * 4];
    __shared__ ff s_row0[4];                            // nu, R_00, (A x)_0 of the start, 1 / nu
    __shared__ ff s_x0;                                 // x_0 at the end (CL: from CTA 0)
    __shared__ double s_sc[8];
    __shared__ float s_drms;
    __shared__ int s_nzr[32], s_flag, s_zero, s_late[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (ms->done || st->status) return;
    unsigned rank = 0, C = 1;
    if (CL) {
        rank = cg::this_cluster().block_rank();
        C = cg::this_cluster().num_blocks();
    }
    const int m = ms->m_sel, n1 = m + 1;
    // this CTA's rows of R (absolute indices [a0, a1)); one CTA: all
    const int a0 = CL ? (int)rank * crows : 0, a1 = CL ? min(a0 + crows, n1) : n1;
    constexpr bool in_smem = CL || SM;
    // the state scalars, loaded (thread 0) ahead of the sums; read after the barriers below
    __shared__ dd s_mu0, s_al0, s_sc0;
    __shared__ long long s_nnz0;
    if (tid == 0) { s_mu0 = ms->mu; s_al0 = ms->alpha; s_sc0 = ms->scale; s_nnz0 = ms->nnz_c; }
    int hf = 0, hff = 0;
    const int L = eig_len(n1), nq = L / 4;
    const int nown = a1 > a0 ? a1 - a0 : 0;             // rows held here
    // (the layout uses crows, the same in every CTA of a cluster, so that an array's offset, which
    // the other CTAs' writes address, does not depend on this CTA's own number of rows)
    float *sh = sm, *sl = sm + (size_t)crows * ldr;
    // 0. start the copy of this CTA's rows of R (hi and lo) into shared memory: one bulk copy per
    //    array (R is row-major with stride ldr), issued by thread 0 after arming the barrier; it
    //    completes behind steps 1 and 2
    __shared__ unsigned long long s_bar;
    if (in_smem && tid == 0 && nown > 0) {
        const unsigned bytes = (unsigned)nown * (unsigned)ldr * 4u;
        mbar_init_arm(&s_bar, 2u * bytes);
        bulk_g2s(sh, Rh + (size_t)a0 * ldr, bytes, &s_bar);
        bulk_g2s(sl, Rl + (size_t)a0 * ldr, bytes, &s_bar);
    }
    // R in global memory: two stage buffers for the streamed products, their barriers armed later
    __shared__ unsigned long long s_sbar[2];
    unsigned spar[2] = {0u, 0u};
    if (!in_smem && tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_sbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_sbar[1])) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    float *vec = in_smem ? sm + 2 * (size_t)crows * ldr : sm;
    float *xs = vec;                                    // float-float x (2 L floats)
    float *ws = vec + 2 * L;                            // FP32 w (L floats)
    double *zd = reinterpret_cast<double *>(vec + 3 * L);   // z (L doubles); first the start's A x (float-float)
    float *hs = vec + 5 * L;                            // the start's H_II c_I (float-float, 2 L floats)
    float *ys = vec + 7 * L;                            // streamed products' results (2 L floats)
    float *stg = vec + 9 * L;                           // stage buffers
    const int srows = eig_stage_rows(n1);

    // 1. sums over I (FP64): c.c, c.b, c.H_II c, |diag H_II|^2, nonzeros (thread t: coordinates
    //    t, t + blockDim, ...; the warps holding one); the coordinates' start values (float-float,
    //    from k_mc_prepare) staged at their absolute index i + 1
    const int nsw = (min(m, (int)blockDim.x) + 31) >> 5;
    double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
    int nzc = 0;
    for (int t = tid; t < m; t += blockDim.x) {
        const double c0 = cI[t], bt = bI[t], ht = HIIc[t], hd = Hdiag[t];
        p0 = fma(c0, c0, p0); p1 = fma(c0, bt, p1); p2 = fma(c0, ht, p2); p3 = fma(hd, hd, p3);
        nzc += (__double_as_longlong(c0) << 1) != 0 ? 1 : 0;
        const float4 f0 = rowf[2 * t], f1 = rowf[2 * t + 1];
        const int a = t + 1;
        xs[2 * a] = f0.x; xs[2 * a + 1] = f0.y;         // c_i
        float *az = reinterpret_cast<float *>(zd);
        az[2 * a] = f0.z; az[2 * a + 1] = f0.w;         // b_i
        hs[2 * a] = f1.x; hs[2 * a + 1] = f1.y;         // (H_II c_I)_i
    }
    if (warp < nsw) {
        const double t = wsum4(p0, p1, p2, p3);
        const int nzw = __reduce_add_sync(0xffffffffu, nzc);
        if ((lane & 7) == 0) s_red[warp * 4 + (lane >> 3)] = t;
        if (lane == 0) s_nzr[warp] = nzw;
    }
    for (int t = n1 + tid; t < L; t += blockDim.x) { xs[2 * t] = 0.0f; xs[2 * t + 1] = 0.0f; ws[t] = 0.0f; }
    if (tid == 0) { xs[0] = 0.0f; xs[1] = 0.0f; ws[0] = 0.0f; }
    __syncthreads();
    // 2. warp 0: the four sums (lane 8 k + j adds value k of warps j, j + 8, ..., then a
    //    three-level butterfly); nu^2 = mu - c.c (lane 0), nu^2 R_00 = alpha - 2 c.b + c.H c
    //    (lane 1) and nu (A x)_0 = alpha - c.b (lane 2) as compensated sums (TwoSum), all three
    //    in the same instructions; the degenerate case (c has no support outside I); 1 / nu in
    //    float-float (Newton) while nu^2 is a normal FP32 number, else by the FP64 rsqrt; then
    //    nu, R_00 and (A x)_0 (float-float).  Tests on FP64 values are integer tests of their bits.
    if (warp == 0) {
        double t = 0.0;
        for (int q = lane & 7; q < nsw; q += 8) t += s_red[q * 4 + (lane >> 3)];
        t += __shfl_xor_sync(0xffffffffu, t, 4);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        const double cc = __shfl_sync(0xffffffffu, t, 0), cb = __shfl_sync(0xffffffffu, t, 8);
        const double chc = __shfl_sync(0xffffffffu, t, 16), hh = __shfl_sync(0xffffffffu, t, 24);
        int nz = 0;
        for (int q = 0; q < nsw; ++q) nz += s_nzr[q];
        const dd a = lane == 0 ? s_mu0 : s_al0;
        const double p = lane == 0 ? -cc : (lane == 1 ? -2.0 * cb : -cb);
        const double q = lane == 1 ? chc : 0.0;
        const dd s1 = dd_two_sum(a.hi, p), s2 = dd_two_sum(s1.hi, q);
        const double r = s2.hi + ((s1.lo + s2.lo) + a.lo);
        const double nu2 = __shfl_sync(0xffffffffu, r, 0);
        const long long nb = __double_as_longlong(nu2);
        const bool deg = (nz >= s_nnz0) || nb <= 0;     // nu^2 <= 0
        const int ex = (int)((nb >> 52) & 0x7ff) - 1023;
        const ff rf = ff_from_double(r), n2f = {__shfl_sync(0xffffffffu, rf.hi, 0), __shfl_sync(0xffffffffu, rf.lo, 0)};
        ff inu_f = {0.0f, 0.0f};
        if (!deg) {
            if (ex > -120 && ex < 120) inu_f = ff_rsqrt(n2f);
            else inu_f = ff_from_double(rsqrt(nu2));
        }
        // lane 0: nu = nu^2 / nu, lane 1: R_00, lane 2: (A x)_0, lane 3: 1 / nu
        const ff yf = lane == 3 ? inu_f : ff_mul(ff_mul(rf, inu_f), lane == 1 ? inu_f : ff{1.0f, 0.0f});
        if (lane < 4) s_row0[lane] = yf;
        const float r00 = __shfl_sync(0xffffffffu, yf.hi, 1);
        if (lane == 0) {
            s_sc[0] = deg ? 1.0 : 0.0;
            s_zero = (deg && __double_as_longlong(cc) <= 0) ? 1 : 0;   // c = 0: no start vector
            const float nf = (float)(m + (deg ? 0 : 1));
            s_drms = sqrtf((__double2float_rn(hh) + (deg ? 0.0f : r00 * r00)) / nf);
        }
    }
    // the copy of R: a bounded wait; a copy that never lands is an error (its bytes may still be in
    // flight: the threads that gave up wait once more, bounded, before the block leaves).  In a
    // cluster the decision is shared, so that every CTA leaves or none.
    const bool late = in_smem && nown > 0 && !mbar_wait0(&s_bar, 1 << 22);
    bool any_late = __syncthreads_or(late);             // scalars, and this block's copy of R, complete
    if (CL) {
        if (tid == 0) {
            cg::cluster_group cl = cg::this_cluster();
            for (unsigned r = 0; r < C; ++r) cl.map_shared_rank(s_late, r)[rank] = any_late ? 1 : 0;
        }
        cg::this_cluster().sync();
        any_late = false;
        for (unsigned r = 0; r < C; ++r) any_late |= s_late[r] != 0;
    }
    if (any_late) {
        if (tid == 0) set_status(st, kErrTimeout);
        if (late) mbar_wait0(&s_bar, 1 << 22);
        return;
    }
    const bool deg = s_sc[0] != 0.0;
    const int off = deg ? 1 : 0;
    const int n = n1 - off;                             // active size
    // row and column 0 of R: R_0i = (b_i - (H_II c_I)_i) / nu (zero when not active); column 0 for
    // this CTA's rows, row 0 where it is held.  They are first read by the product A w after the
    // barriers of the first sums below.
    {
        float *Wh = in_smem ? sh : Rh, *Wl = in_smem ? sl : Rl;
        const ff inu = s_row0[3];
        for (int t = tid; t < m; t += blockDim.x) {
            const int a = t + 1;
            const bool col = a >= a0 && a < a1, row = a0 == 0 && nown > 0;
            if (!col && !row) continue;
            const float4 f1 = rowf[2 * t + 1];
            const ff r0 = deg ? ff{0.0f, 0.0f} : ff_mul(ff{f1.z, f1.w}, inu);
            if (row) { Wh[a] = r0.hi; Wl[a] = r0.lo; }
            if (col) { Wh[(size_t)(a - a0) * ldr] = r0.hi; Wl[(size_t)(a - a0) * ldr] = r0.lo; }
        }
        if (tid == 0 && a0 == 0 && nown > 0) {
            const ff r00 = deg ? ff{0.0f, 0.0f} : s_row0[1];
            Wh[0] = r00.hi; Wl[0] = r00.lo;
        }
    }
    // (in global memory, the streamed products read them through the TMA unit: order these writes
    // before its reads; a barrier follows before the first product)
    if (!in_smem) asm volatile("fence.proxy.async.global;" ::: "memory");

    // 3. the start: thread group `lr` of tpr threads takes absolute row ra = a0 + lr (active from
    //    off); the group's first lane (lead) speaks for the row in sums.  x = [nu; c_I] (not
    //    normalised) and A x in closed form; degenerate: x = c_I, A x = H_II c_I; c = 0 (not
    //    reached in practice): x = e_off with A x computed
    const int lr = tid / tpr, kk = tid - lr * tpr;
    const int ra = a0 + lr;
    const bool act = ra >= off && ra < a1, lead = act && kk == 0;
    const bool zero_start = s_zero != 0;
    ff x = {0.0f, 0.0f}, ax = {0.0f, 0.0f};
    float d = 0.0f;
    if (act) {
        if (zero_start) {
            x = ff{ra == off ? 1.0f : 0.0f, 0.0f};
        } else if (ra == 0) {
            x = s_row0[0];
            ax = s_row0[2];
        } else {
            x = ff{xs[2 * ra], xs[2 * ra + 1]};
            const float *az = deg ? hs : reinterpret_cast<const float *>(zd);
            ax = ff{az[2 * ra], az[2 * ra + 1]};
        }
        d = ra == 0 ? s_row0[1].hi : (in_smem ? sh[(size_t)lr * ldr + ra] : Rh[(size_t)ra * ldr + ra]);
    }
    float pv = 0.0f, apv = 0.0f;                        // search direction p and A p
    bool have_p = false;
    ff theta = {0.0f, 0.0f}, xx = {1.0f, 0.0f};
    float best = 3.0e38f;
    int stall = 0, it = 0;
    const float drms = s_drms;                          // RMS of diag A, a scale for the tests below
    // A x follows x implicitly (x <- yx x + yw w + yp p gives A x <- yx A x + yw A w + yp A p, the
    // last two in FP32) and is recomputed exactly each time the residual falls below `refresh`
    // (relative), and always before convergence is accepted: an implicit A x drifts by about the
    // FP32 rounding of the steps taken since the last exact one (and the closed-form start's by
    // the float-float rounding of R)
    bool exact = false, want_exact = zero_start;
    float refresh = 1e-12f;                             // (relative |r|^2: |r| below 1e-6 of the scale)
    for (;; ++it) {
        // A x recomputed exactly for the current x when asked for (x gathered in full first)
        if (want_exact) {
            if (lead) {
                if (CL) {
                    cg::cluster_group cl = cg::this_cluster();
                    for (unsigned r = 0; r < C; ++r) {
                        float *d2 = cl.map_shared_rank(xs, r);
                        d2[2 * ra] = x.hi; d2[2 * ra + 1] = x.lo;
                    }
                } else {
                    xs[2 * ra] = x.hi; xs[2 * ra + 1] = x.lo;
                }
            }
            if (CL) cg::this_cluster().sync(); else __syncthreads();
            if constexpr (in_smem) {
                ax = ff_row(sh, sl, ldr, nq, lr, kk, tpr, act, xs);
            } else {
                eig_stream<true>(Rh, Rl, ldr, n1, nq, stg, srows, s_sbar, spar, xs, ys, st);
                ax = act ? ff{ys[2 * ra], ys[2 * ra + 1]} : ff{0.0f, 0.0f};
            }
            exact = true;
            want_exact = false;
        }
        // (a) theta = x.Ax / x.x, r = A x - theta x
        {
            ff t[2] = {lead ? ff_mul(x, ax) : ff{0.0f, 0.0f}, lead ? ff_mul(x, x) : ff{0.0f, 0.0f}};
            bsum_ff<CL, 2>(t, s_rff, hff, rank, C);
            xx = t[1];
            theta = ff_div(t[0], t[1]);
        }
        const float r = act ? ff_to_float(ff_add(ax, ff_neg(ff_mul(theta, x)))) : 0.0f;
        const float th = ff_to_float(theta);
        const float scale = fmaxf(fabsf(th), drms);
        // (b) preconditioned residual w = r / |A_ii - theta| (the absolute value keeps the
        //     preconditioner positive definite while theta is still above some diagonal entries;
        //     an indefinite one stalls the iteration)
        const float den = fmaxf(fabsf(d - th), 1e-4f * fmaxf(scale, 1e-30f));
        float wv = act ? __fdividef(r, den) : 0.0f;
        const float xh = x.hi;
        float red[3] = {lead ? r * r : 0.0f, lead ? xh * wv : 0.0f, lead ? xh * pv : 0.0f};
        bsum_f<CL, 3>(red, s_rf, hf, rank, C);
        const float nres2 = red[0];                     // |r|^2; the tests below compare squares
        const float sc2 = scale * scale;
        // stop at the float-float floor, at the cap, or when progress has ended well below it;
        // only a residual of an exact A x ends the iteration: with an implicit one the step below
        // is taken and A x is recomputed at the start of the next iteration (likewise once the
        // residual is below `refresh`, which then moves down five decades: the steps after a
        // refresh are about the residual's size, so the implicit A x drifts by about 1e-7 of it)
        if (nres2 < best * 0.49f) { best = nres2; stall = 0; } else ++stall;
        const bool stop = !(nres2 > 1e-28f * sc2 * (float)n) || it >= kEigMaxIt || (stall >= 4 && nres2 < 1e-22f * sc2);
        if (stop && exact) break;
        if (!exact && (stop || nres2 < refresh * sc2)) {
            want_exact = true;
            refresh = fminf(refresh, __fdividef(nres2, fmaxf(sc2, 1e-30f))) * 1e-10f;   // five decades of |r|
            if (stop) { best = 3.0e38f; stall = 0; }
        }
        // w and p orthogonalised against x (A p likewise, with A x as held)
        const float ixx = __fdividef(1.0f, ff_to_float(xx));
        wv -= red[1] * ixx * xh;
        if (have_p) {
            pv -= red[2] * ixx * xh;
            apv -= red[2] * ixx * ff_to_float(ax);
        }
        // (c) A w (w gathered in full first)
        if (lead) {
            if (CL) {
                cg::cluster_group cl = cg::this_cluster();
                for (unsigned r2 = 0; r2 < C; ++r2) cl.map_shared_rank(ws, r2)[ra] = wv;
            } else {
                ws[ra] = wv;
            }
        }
        if (CL) cg::this_cluster().sync(); else __syncthreads();
        float awv;
        if constexpr (in_smem) {
            awv = f_row(sh, ldr, nq, lr, kk, tpr, act, ws);
        } else {
            eig_stream<false>(Rh, Rl, ldr, n1, nq, stg, srows, s_sbar, spar, ws, ys, st);
            awv = act ? ys[ra] : 0.0f;
        }
        // (d) projections on span{x, w, p}, the pencil shifted by theta: its x row is
        //     (A x - theta x) . [x, w, p] = [0, r.w, r.p]
        const float aws = awv - th * wv, aps = apv - th * pv;
        float pr[8] = {r * wv, r * pv, wv * aws, wv * aps, pv * aps, wv * wv, wv * pv, pv * pv};
        if (!lead)
#pragma unroll
            for (int q = 0; q < 8; ++q) pr[q] = 0.0f;
        bsum_f<CL, 8>(pr, s_rf, hf, rank, C);
        // Rayleigh-Ritz: the lowest eigenpair of (P - mu G) y = 0 with P = [0 rw rp; rw sww swp;
        // rp swp spp] and the Gram matrix G (x orthogonal to w and p), by the Cholesky factor L of
        // G: C = L^-1 P L^-T, y = L^-T v
        const float rw = pr[0], rp = pr[1], sww = pr[2], swp = pr[3], spp = pr[4];
        const float gxx = ff_to_float(xx), gxw = 0.0f, gxp = 0.0f, gww = pr[5], gwp = pr[6], gpp = pr[7];
        float yx = 1.0f, yw = 0.0f, yp = 0.0f;
        const float il00 = rsqrtf(gxx);                 // L = [l00 0 0; l10 l11 0; l20 l21 l22], inverses of its diagonal
        const float l10 = gxw * il00, l20 = gxp * il00;
        const float d11 = gww - l10 * l10;
        if (d11 > 1e-12f * gww && gww > 0.0f) {
            const float il11 = rsqrtf(d11);
            bool use_p = have_p && gpp > 0.0f;
            float l21 = 0.0f, il22 = 0.0f;
            if (use_p) {
                l21 = (gwp - l20 * l10) * il11;
                const float d22 = gpp - l20 * l20 - l21 * l21;
                use_p = d22 > 1e-6f * gpp;
                if (use_p) il22 = rsqrtf(d22);
            }
            // M = L^-1 P (rows), then C = M L^-T
            const float m00 = 0.0f, m01 = rw * il00, m02 = rp * il00;
            const float m10 = (rw - l10 * m00) * il11, m11 = (sww - l10 * m01) * il11, m12 = (swp - l10 * m02) * il11;
            const float c00 = m00 * il00;
            const float c01 = (m01 - l10 * c00) * il11;
            const float c11 = (m11 - l10 * (m10 * il00)) * il11;
            float v0, v1, v2 = 0.0f, lam;
            if (use_p) {
                const float m20 = (rp - l20 * m00 - l21 * m10) * il22;
                const float m21 = (swp - l20 * m01 - l21 * m11) * il22;
                const float m22 = (spp - l20 * m02 - l21 * m12) * il22;
                const float c02 = (m02 - l20 * c00 - l21 * c01) * il22;
                const float c12 = (m12 - l20 * (m10 * il00) - l21 * c11) * il22;
                const float c22 = (m22 - l20 * (m20 * il00) - l21 * ((m21 - l10 * (m20 * il00)) * il11)) * il22;
                sym3_lowest(c00, c01, c02, c11, c12, c22, lam, v0, v1, v2);
                yp = v2 * il22;
                yw = (v1 - l21 * yp) * il11;
                yx = (v0 - l10 * yw - l20 * yp) * il00;
            } else {
                sym2_lowest(c00, c01, c11, lam, v0, v1);
                yw = v1 * il11;
                yx = (v0 - l10 * yw) * il00;
                yp = 0.0f;
            }
            if (yx < 0.0f) { yx = -yx; yw = -yw; yp = -yp; }
        }
        // (e) x <- yx x + yw w + yp p, A x likewise; p <- yw w + yp p (unit length), A p likewise
        const float np = yw * wv + yp * pv;
        const float nap = yw * awv + yp * apv;
        const float pn2 = yw * yw * gww + 2.0f * yw * yp * gwp + yp * yp * gpp;
        x = ff_add(ff_mul_f(x, yx), ff{np, 0.0f});
        ax = ff_add(ff_mul_f(ax, yx), ff{nap, 0.0f});
        exact = false;
        if (pn2 > 0.0f) {
            const float ip = rsqrtf(pn2);
            pv = np * ip;
            apv = nap * ip;
            have_p = true;
        } else {
            pv = 0.0f; apv = 0.0f; have_p = false;
        }
    }
    // 4. z = zs x, zs = sqrt(-lambda / x.x) (float-float); the reduced problem needs lambda < 0
    //    (theta is the same in every CTA, so all return together)
    if (!(theta.hi < 0.0f || (theta.hi == 0.0f && theta.lo < 0.0f))) {
        if (tid == 0 && rank == 0) set_status(st, kErrNotNegative);
        return;
    }
    const ff q = ff_div(ff_neg(theta), xx);
    const ff zs_f = ff_mul(q, ff_rsqrt(q));
    if (lead) zd[ra] = ff_to_double(x);
    // x_0 (row 0, with CTA 0's thread 0) to every CTA
    if (tid == 0 && rank == 0) {
        if (CL) {
            cg::cluster_group cl = cg::this_cluster();
            for (unsigned r = 0; r < C; ++r) *cl.map_shared_rank(&s_x0, r) = x;
        } else {
            s_x0 = x;
        }
    }
    if (CL) cg::this_cluster().sync(); else __syncthreads();
    // sign (Eq. def-z wants gamma >= 0): z_0 >= 0; degenerate or z_0 = 0: z . c_I >= 0, the FP64 dot
    // taken only then; gamma = z_0 / nu (every CTA the same)
    if (tid == 0) {
        const ff z0 = deg ? ff{0.0f, 0.0f} : ff_mul(zs_f, s_x0);
        s_flag = (deg || z0.hi == 0.0f) ? 1 : 0;
        s_sc[3] = z0.hi < 0.0f ? -1.0 : 1.0;
        const ff g = ff_mul(ff{fabsf(z0.hi), z0.hi < 0.0f ? -z0.lo : z0.lo}, s_row0[3]);
        s_sc[4] = deg ? 1.0 : ff_to_double(g);
        s_sc[5] = ff_to_double(zs_f);
    }
    __syncthreads();
    if (s_flag) {                                       // uniform over the cluster: s_flag agrees
        const double dot = csum_d<CL>(lead && ra >= 1 ? zd[ra] * cI[ra - 1] : 0.0, s_red, rank, C);
        if (tid == 0) s_sc[3] = dot < 0.0 ? -1.0 : 1.0;
        __syncthreads();
    }
    const double sgn = s_sc[3], gamma = s_sc[4], zs = s_sc[5];
    const bool bad = !isfinite(gamma) || !(gamma > 1e-200);
    // 5. eta (Eq. def-z) and the compression thresholds (the lead of row i + 1: coordinate i), while
    //    thread 0 forms the new scale s' = s gamma (double-double) and 1 / s'
    const bool coord = lead && ra >= 1;
    const int ic = ra - 1;
    double eta = 0.0, zn = 0.0, ct = 0.0;
    if (coord) {
        ct = cI[ic];                                    // reloaded: nothing of step 1 stays live in the loop
        zn = sgn * (zd[ra] * zs);
        eta = zn - gamma * ct;
        etaout[ic] = eta;
        thr[ic] = eta != 0.0 ? P.tau / fabs(eta) : 1.0e308;
    }
    if (tid == 0) {
        const dd s_new = dd_mul_d(s_sc0, gamma);
        s_sc[6] = 1.0 / s_new.hi;
        if (rank == 0) {
            ms->pend_scale = s_new;
            ms->pend_gamma = gamma;
            ms->pend_it = it;
            ms->pend_deg = deg ? 1 : 0;
            ms->n_cand = 0;                             // the scatter builds the next candidate list
            if (bad) set_status(st, kErrNonfinite);
        }
    }
    __syncthreads();
    // 6. the scatter weights and the new stored c_I; the change in nonzeros of c
    const double rsc = s_sc[6];
    bool to = false, from = false;
    if (coord) {
        w[ic] = eta * rsc;
        if (!bad) {
            P.table[sel[ic].slot].c = zn * rsc;
            cnz_set(P, sel[ic].A, sel[ic].B);
        }
        from = ct != 0.0 && zn == 0.0;
        to = ct == 0.0 && zn != 0.0;
    }
    const int dn = __popc(__ballot_sync(0xffffffffu, to)) - __popc(__ballot_sync(0xffffffffu, from));
    if (lane == 0 && dn != 0 && !bad) atomicAdd(reinterpret_cast<unsigned long long *>(&ms->nnz_c),
                                                (unsigned long long)(long long)dn);
}

// ---------------------------------------------------------------------------
// The scalars of Alg. 2's update of c (one block, inside the scatter's launch,
// so that it runs beside the scatter): with gamma and eta from k_mc_eigen,
//   mu'    = gamma^2 mu + 2 gamma eta.c_I + eta.eta,
//   alpha' = gamma^2 alpha + 2 gamma eta.b_I + eta^T H_II eta   (double-double),
// eta^T H_II eta in float-float from R's rows and columns 1..m; the energy
// alpha / mu, the dx rule, the new scale, the counters.
// ---------------------------------------------------------------------------
struct McUpdate {
    const double *cI, *bI, *eta;
    const float *Rh, *Rl;
    int ldr, on;                    // on = 0: no update block (the scatter of a start vector)
};
__device__ void mc_update_block(const Problem &P, McState *ms, IterState *st, const double *cI, const double *bI,
                                const double *etaout, const float *Rh, const float *Rl, int ldr, int m,
                                float *s_eta, double *s_red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int L = eig_len(m + 1), nq = L / 4;
    // eta as float-float in R's absolute indexing (entry 0 and the padding are zero)
    for (int a = tid; a < L; a += blockDim.x) {
        const ff e = (a >= 1 && a <= m) ? ff_from_double(etaout[a - 1]) : ff{0.0f, 0.0f};
        s_eta[2 * a] = e.hi;
        s_eta[2 * a + 1] = e.lo;
    }
    // FP64 sums eta.c_I, eta.b_I, eta.eta (threads over coordinates)
    double ec = 0.0, eb = 0.0, ee = 0.0;
    for (int i = tid; i < m; i += blockDim.x) {
        const double e = etaout[i];
        ec = fma(e, cI[i], ec);
        eb = fma(e, bI[i], eb);
        ee = fma(e, e, ee);
    }
    __syncthreads();
    // eta^T H_II eta over R's rows and columns 1..m: warp w takes the row pairs (a, a + nw),
    // a = 1 + w, 1 + w + 2 nw, ...; lane l the 4-column chunks l, l + 32, ... of both rows
    const float4 *e4 = reinterpret_cast<const float4 *>(s_eta);
    float ah = 0.0f, al = 0.0f;
    for (int a = 1 + warp; a <= m; a += 2 * nw) {
        const int b = a + nw;
        const bool two = b <= m;
        const float4 *h0 = reinterpret_cast<const float4 *>(Rh + (size_t)a * ldr);
        const float4 *l0 = reinterpret_cast<const float4 *>(Rl + (size_t)a * ldr);
        const float4 *h1 = reinterpret_cast<const float4 *>(Rh + (size_t)(two ? b : a) * ldr);
        const float4 *l1 = reinterpret_cast<const float4 *>(Rl + (size_t)(two ? b : a) * ldr);
        float th0 = 0.0f, tl0 = 0.0f, th1 = 0.0f, tl1 = 0.0f;
        for (int q = lane; q < nq; q += 32) {
            const float4 hv0 = h0[q], lv0 = l0[q], hv1 = h1[q], lv1 = l1[q];
            const float4 xa = e4[2 * q], xb = e4[2 * q + 1];
            ff_mac(th0, tl0, hv0.x, lv0.x, ff{xa.x, xa.y});
            ff_mac(th0, tl0, hv0.y, lv0.y, ff{xa.z, xa.w});
            ff_mac(th0, tl0, hv0.z, lv0.z, ff{xb.x, xb.y});
            ff_mac(th0, tl0, hv0.w, lv0.w, ff{xb.z, xb.w});
            ff_mac(th1, tl1, hv1.x, lv1.x, ff{xa.x, xa.y});
            ff_mac(th1, tl1, hv1.y, lv1.y, ff{xa.z, xa.w});
            ff_mac(th1, tl1, hv1.z, lv1.z, ff{xb.x, xb.y});
            ff_mac(th1, tl1, hv1.w, lv1.w, ff{xb.z, xb.w});
        }
        ff t = ff_mul(ff_norm(th0, tl0), ff{s_eta[2 * a], s_eta[2 * a + 1]});
        if (two) t = ff_add(t, ff_mul(ff_norm(th1, tl1), ff{s_eta[2 * b], s_eta[2 * b + 1]}));
        const ff u = ff_two_sum(ah, t.hi);
        ah = u.hi;
        al = __fadd_rn(al, __fadd_rn(u.lo, t.lo));
    }
    ff eh = ff_norm(ah, al);
    for (int o = 16; o > 0; o >>= 1) {
        eh = ff_add(eh, ff{__shfl_down_sync(0xffffffffu, eh.hi, o), __shfl_down_sync(0xffffffffu, eh.lo, o)});
        ec += __shfl_down_sync(0xffffffffu, ec, o);
        eb += __shfl_down_sync(0xffffffffu, eb, o);
        ee += __shfl_down_sync(0xffffffffu, ee, o);
    }
    if (lane == 0) {
        s_red[4 * warp] = ec; s_red[4 * warp + 1] = eb; s_red[4 * warp + 2] = ee;
        reinterpret_cast<ff *>(s_red + 4 * warp + 3)[0] = eh;
    }
    __syncthreads();
    if (warp != 0) return;
    // warp 0: the warps' sums in order (every lane), then mu' (lane 0) and alpha' (lane 1) in the same
    // instructions, double-double
    double sc = 0.0, sb = 0.0, se = 0.0;
    ff sh = {0.0f, 0.0f};
    for (int q = 0; q < nw; ++q) {
        sc += s_red[4 * q]; sb += s_red[4 * q + 1]; se += s_red[4 * q + 2];
        sh = ff_add(sh, reinterpret_cast<const ff *>(s_red + 4 * q + 3)[0]);
    }
    const dd mu0 = ms->mu, al0 = ms->alpha;
    const double gamma = ms->pend_gamma;
    const bool a1 = lane == 1;
    const dd g2 = dd_two_prod(gamma, gamma);
    const dd out = dd_add(dd_add(dd_mul(g2, a1 ? al0 : mu0), dd_two_prod(2.0 * gamma, a1 ? sb : sc)),
                          dd{a1 ? ff_to_double(sh) : se, 0.0});
    const dd al_n = {__shfl_sync(0xffffffffu, out.hi, 1), __shfl_sync(0xffffffffu, out.lo, 1)};
    const double dxr = sqrt(se);
    if (lane != 0) return;
    const dd mu_n = out, s_new = ms->pend_scale;
    const double dx0 = ms->dx;
    const long long its = ms->iterations, eit = ms->eig_iters_total;
    const int it = ms->pend_it, deg = ms->pend_deg;
    const bool ok = isfinite(mu_n.hi) && isfinite(al_n.hi);
    const dd mu_k = ok ? mu_n : mu0, al_k = ok ? al_n : al0;
    if (!ok) {
        set_status(st, kErrNonfinite);
    } else {
        ms->mu = mu_n;
        ms->alpha = al_n;
        ms->scale = s_new;
        st->scale = s_new;
    }
    const double dxn = P.theta * dx0 + (1.0 - P.theta) * dxr;
    ms->energy = dd_div_to_d(al_k, mu_k);
    ms->iterations = its + 1;
    ms->dx = dxn;
    if (P.dx_threshold > 0.0 && dxn < P.dx_threshold) ms->done_pending = 1;
    ms->degenerate = deg;
    ms->last_gamma = gamma;
    ms->eig_iters = it;
    ms->eig_iters_total = eit + it;
}

// ---------------------------------------------------------------------------
// b += H_{:,I} eta for the m columns (stored units), gather, candidates.
//
// Work items of one warp each.  The off-diagonal elements of a column are
// products of single excitations of its determinant: an opposite-spin double
// is an alpha single times a beta single, a same-spin double an occupied pair
// times a virtual pair of one string.  An item gives every lane one factor,
// kept in registers, and runs the other factor over a short range, one
// uniform (broadcast) load per step:
//   AB item: 32 beta singles (one per lane) x kAbChunk alpha singles; the
//            element is the integral at the sum of the two entries' offsets,
//            its key the two changed strings, its hash the xor of their hashes;
//   AA / BB: 32 virtual pairs x kSsChunk occupied pairs of one string;
//   S item:  32 singles, each summing its terms in the order of Eq. (entry).
// The column's single-excitation entries and orbital lists are built once per
// iteration (k_mc_prepare, k_mc_start).  Warps take items of all columns from
// a global counter; each item leaves one gather partial (sum_j H_ji c_j over
// its elements), which k_mc_finalize adds per column in item order.  An item
// first evaluates its elements; those that need the table (|H| at or above
// the column's threshold, or c_j possibly nonzero by the filter) go to the
// warp's queue, which the warp then looks up 64 at a time, two per lane with
// both first slots in flight (one call site of the lookup routine for every
// item kind keeps the kernel's code small).
// ---------------------------------------------------------------------------
constexpr int kWarpCand = 192;      // per-warp buffer of new candidates (flushed above kWarpCand - 32 kDrainU)

// L2 eviction priorities for the scatter: a table slot's last touch in a lookup
// is the add to b (evict first after it; the slot's load keeps the normal
// priority so that the line is still in L2 when the add arrives), while the
// integrals, the c != 0 filter and the candidate marks are read by every
// element and must stay in L2 (evict last).
__device__ __forceinline__ unsigned long long l2_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_evict_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ double ldg_keep(const double *p, unsigned long long pol) {
    double x;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(x) : "l"(p), "l"(pol));
    return x;
}
__device__ __forceinline__ unsigned ldg_keep(const unsigned *p, unsigned long long pol) {
    unsigned x;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(x) : "l"(p), "l"(pol));
    return x;
}
__device__ __forceinline__ void red_add_hint(double *p, double v, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
// candidate mark of slot s (true if this call set it), kept in L2
__device__ __forceinline__ bool mark_set_keep(const Problem &P, long long s, unsigned long long pol) {
    const unsigned bit = 1u << (unsigned)(s & 31);
    unsigned old;
    asm volatile("atom.global.or.L2::cache_hint.b32 %0, [%1], %2, %3;"
                 : "=r"(old)
                 : "l"(P.mark + (s >> 5)), "r"(bit), "l"(pol)
                 : "memory");
    return !(old & bit);
}

// The whole 32-byte slot {A, B, c, b} in one load: one DRAM access for the key
// and the values (two 16-byte loads of one slot cost two accesses of random
// slots on this memory system).  L2 only, re-read on every call.
__device__ __forceinline__ void ld_slot(const Slot *s, unsigned long long &ka, unsigned long long &kb, double &c) {
    unsigned long long cb;
    [[maybe_unused]] unsigned long long bb;
    asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(ka), "=l"(kb), "=l"(cb), "=l"(bb)
                 : "l"(s));
    c = __longlong_as_double((long long)cb);
}

// Probe for {a, b} whose first slot (at pos) the caller has loaded: key (ka,
// kb) and c (sc).  Returns the slot, or -1 (absent, not inserted) / -2 (error,
// status set).  c: the slot's stored c.
__device__ __forceinline__ long long mc_resolve(const Problem &P, IterState *st, unsigned long long a,
                                                unsigned long long b, unsigned long long pos, unsigned long long ka,
                                                unsigned long long kb, double sc, bool insert, bool &inserted,
                                                double &c) {
    const bool both_nonzero = (P.na > 0) && (P.nb > 0);
    for (int probe = 0; probe < P.max_probe; ++probe) {
        Slot *s = P.table + pos;
        if (probe > 0) ld_slot(s, ka, kb, sc);
        int spins = 0;
        while (both_nonzero && ((ka == 0ull) != (kb == 0ull))) {     // an insert in flight
            if (++spins > (1 << 20)) { set_status(st, kErrTimeout); return -2; }
            ld_slot(s, ka, kb, sc);
        }
        if (ka == a && (kb & kKeyMaskB) == b) {
            c = sc;
            return (long long)pos;
        }
        if (ka == 0ull && kb == 0ull) {
            if (!insert) return -1;
            unsigned long long oa, ob;
            cas128(&s->a, 0ull, 0ull, a, b, oa, ob);
            if (oa == 0ull && ob == 0ull) {
                inserted = true;
                c = 0.0;
                return (long long)pos;
            }
            if (oa == a && (ob & kKeyMaskB) == b) {      // lost to an insert of the same key
                c = __ldcg(&s->c);
                return (long long)pos;
            }
        }
        pos = (pos + 1) & P.mask;
    }
    set_status(st, kErrTableFull);
    return -2;
}

// Per-warp scatter context: the column's constants, counters and the lookup queue.
struct McWarp {
    unsigned long long *qa, *qb, *qh;
    double *qH;
    long long *wcand;
    unsigned long long pol_first, pol_last;        // L2 eviction policies: table slots / hot structures
    unsigned long long tib;
    double wi, gather;
    int qn, nwc, c_el, c_app, c_drop, c_ins;
    bool err;
};

// filter word of hash h (the c != 0 bit is bit (h >> 32) & 31 of it); all ones without a filter
__device__ __forceinline__ unsigned cnz_word(const Problem &P, unsigned long long h, unsigned long long pol) {
    return P.cnz ? ldg_keep(P.cnz + (((h >> 32) & P.cnz_mask) >> 5), pol) : 0xffffffffu;
}

// Element (oa, ob) with hash hk and value H (`ok`: this lane holds one) with its filter word cw:
// counted, and queued when it needs the table (|H| >= thr, compared as bit patterns, or c_j
// possibly nonzero); otherwise c_j = 0 and the compression rule drops it here.
__device__ __forceinline__ void mc_push(McWarp &W, bool ok, unsigned long long oa, unsigned long long ob,
                                        unsigned long long hk, double H, unsigned cw) {
    const int lane = threadIdx.x & 31;
    bool need = false;
    if (ok && !is_zero(H)) {
        ++W.c_el;
        need = ((cw >> (unsigned)((hk >> 32) & 31)) & 1u) || abs_bits(H) >= W.tib;
        if (!need) ++W.c_drop;
    }
    const unsigned int nm = __ballot_sync(0xffffffffu, need);
    if (need) {
        const int at = W.qn + __popc(nm & ((1u << lane) - 1u));
        W.qa[at] = oa; W.qb[at] = ob; W.qh[at] = hk; W.qH[at] = H;
    }
    W.qn += __popc(nm);
}

// The warp's candidate buffer to the global list (one reservation); entries
// beyond the list's capacity are not written and set the status.
__device__ __forceinline__ void mc_flush_cand(const Problem &P, McState *ms, IterState *st, long long *wcand, int &nwc,
                                              long long *cand) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    int base = 0;
    if (lane == 0 && nwc > 0) base = atomicAdd(&ms->n_cand, nwc);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < nwc; i += 32) {
        if ((long long)base + i < P.cap_cand) cand[base + i] = wcand[i];
        else set_status(st, kErrInternal);
    }
    nwc = 0;
    __syncwarp();
}

// The queue's lookups, kDrainU per lane at a time (all their first slots in
// flight together): find the slot (insert when the rule passes), add w H to b,
// gather H c, mark the slot as a candidate of the next selection; the lane that
// marks it appends it to the warp's candidate buffer.
constexpr int kDrainU = 2;
__device__ __forceinline__ void mc_drain(const Problem &P, McState *ms, IterState *st, long long *cand, McWarp &W) {
    const int lane = threadIdx.x & 31;
    while (W.qn > 0 && !W.err) {
        __syncwarp();
        const int n = min(W.qn, 32 * kDrainU), base = W.qn - n;
        bool has[kDrainU];
        unsigned long long oa[kDrainU], ob[kDrainU], pos[kDrainU], ka[kDrainU], kb[kDrainU];
        double H[kDrainU], sc[kDrainU];
#pragma unroll
        for (int u = 0; u < kDrainU; ++u) {
            has[u] = lane + 32 * u < n;
            const int at = base + lane + 32 * u;
            oa[u] = has[u] ? W.qa[at] : 0ull;
            ob[u] = has[u] ? W.qb[at] : 0ull;
            pos[u] = has[u] ? (W.qh[at] & P.mask) : 0ull;
            H[u] = has[u] ? W.qH[at] : 0.0;
            ka[u] = kb[u] = 0ull;
            sc[u] = 0.0;
            if (has[u]) ld_slot(P.table + pos[u], ka[u], kb[u], sc[u]);
        }
        __syncwarp();
        W.qn = base;
        bool first[kDrainU];
        long long s[kDrainU];
#pragma unroll
        for (int u = 0; u < kDrainU; ++u) {
            first[u] = false;
            s[u] = -1;
            if (!has[u]) continue;
            const bool big = abs_bits(H[u]) >= W.tib;
            bool ins = false;
            double cj = 0.0;
            s[u] = mc_resolve(P, st, oa[u], ob[u], pos[u], ka[u], kb[u], sc[u], big, ins, cj);
            if (s[u] == -2) {
                W.err = true;
            } else if (s[u] < 0 || !(!is_zero(cj) || big)) {
                ++W.c_drop;
            } else {
                red_add_hint(&P.table[s[u]].bv, W.wi * H[u], W.pol_first);
                ++W.c_app;
                W.c_ins += ins ? 1 : 0;
                W.gather = fma(H[u], cj, W.gather);
                first[u] = mark_set_keep(P, s[u], W.pol_last);
            }
        }
#pragma unroll
        for (int u = 0; u < kDrainU; ++u) {
            const unsigned int fm = __ballot_sync(0xffffffffu, first[u]);
            if (first[u]) W.wcand[W.nwc + __popc(fm & ((1u << lane) - 1u))] = s[u];
            W.nwc += __popc(fm);
        }
        if (W.nwc > kWarpCand - 32 * kDrainU) mc_flush_cand(P, ms, st, W.wcand, W.nwc, cand);
        W.err = __any_sync(0xffffffffu, W.err);
    }
    W.qn = 0;
}

constexpr int kAbChunk = 4;         // alpha singles per opposite-spin item
constexpr int kSsChunk = 4;         // occupied pairs per same-spin item
constexpr int kScatterQ = 32 * 4;   // per-warp queue: one item's elements at most

// Opposite-spin doubles: lane = beta single sb, alpha singles [sa0, sa1), all in flight together.
__device__ __forceinline__ void mc_item_ab(const Problem &P, McWarp &W, const ColEnt *tA, const ColEnt *tB, int nsB,
                                           int sb, int sa0, int sa1) {
    const bool lane_ok = sb < nsB;
    ColEnt eb;
    if (lane_ok) {
        eb = tB[sb];
    } else {
        eb.key = 0ull; eb.h = 0ull; eb.goff = 0; eb.info = 0;
    }
    const int kb = (eb.info >> 24) & 0xff;
    unsigned long long ka[kAbChunk], hk[kAbChunk];
    double H[kAbChunk];
    unsigned cw[kAbChunk];
    bool ok[kAbChunk];
#pragma unroll
    for (int u = 0; u < kAbChunk; ++u) {
        ok[u] = false;
        H[u] = 0.0;
        ka[u] = 0ull;
        hk[u] = 0ull;
        cw[u] = 0u;
        if (sa0 + u < sa1) {
            const ColEnt ea = tA[sa0 + u];                 // uniform: one broadcast load
            ka[u] = ea.key;
            hk[u] = ea.h ^ eb.h;
            ok[u] = lane_ok && k_conserved(P, (ea.info >> 24) & 0xff, kb);
            if (ok[u]) {
                H[u] = apply_parity(ldg_keep(P.g + ea.goff + eb.goff, W.pol_last),
                                    (unsigned long long)((ea.info ^ eb.info) & 1));
                cw[u] = cnz_word(P, hk[u], W.pol_last);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < kAbChunk; ++u) mc_push(W, ok[u], ka[u], eb.key, hk[u], H[u], cw[u]);
}

// Same-spin doubles of one string X (the other string Y with hash hY): lane =
// virtual pair vp, occupied pairs [op0, op1); the element of Eq. (entry) with
// i < j occupied, a < b empty: (ia|jb) - (ib|ja) times the sign of i -> a then
// j -> b.
__device__ __forceinline__ void mc_item_ss(const Problem &P, McWarp &W, bool alpha, unsigned long long X,
                                           unsigned long long Y, unsigned long long hY, const ColLists &L, int vp,
                                           int op0, int op1) {
    const int N = P.N, N2 = N * N;
    const int cv2 = alpha ? P.cva2 : P.cvb2;
    const bool lane_ok = vp < cv2;
    const unsigned char *occ = alpha ? L.occA : L.occB;
    const unsigned char *vir = alpha ? L.virA : L.virB;
    int a = 0, b = 0;
    if (lane_ok) {
        const unsigned short pv = __ldg((alpha ? P.pair_va : P.pair_vb) + vp);
        a = vir[pv & 0xff];
        b = vir[pv >> 8];
    }
    const unsigned short *po_t = alpha ? P.pair_oa : P.pair_ob;
    const int aN2 = a * N2, bN2 = b * N2;
    unsigned long long key[kSsChunk], hk[kSsChunk];
    double H[kSsChunk];
    unsigned cw[kSsChunk];
    bool ok[kSsChunk];
#pragma unroll
    for (int u = 0; u < kSsChunk; ++u) {
        ok[u] = false;
        key[u] = 0ull;
        hk[u] = 0ull;
        H[u] = 0.0;
        cw[u] = 0u;
        if (op0 + u < op1 && lane_ok) {
            const unsigned short po = __ldg(po_t + op0 + u);      // uniform
            const int i = occ[po & 0xff], j = occ[po >> 8];
            const unsigned long long m1 = X & between_mask(i, a);
            const unsigned long long X1 = X ^ (1ull << i) ^ (1ull << a);
            const unsigned long long m2 = X1 & between_mask(j, b);
            key[u] = X1 ^ (1ull << j) ^ (1ull << b);
            hk[u] = (alpha ? hash_alpha(key[u]) : hash_beta(key[u])) ^ hY;
            const int base = i * N * N2 + j * N;
            H[u] = apply_parity(ldg_keep(P.g + base + aN2 + b, W.pol_last) - ldg_keep(P.g + base + bN2 + a, W.pol_last),
                                m1 ^ m2);
            cw[u] = cnz_word(P, hk[u], W.pol_last);
            ok[u] = true;
        }
    }
#pragma unroll
    for (int u = 0; u < kSsChunk; ++u)
        mc_push(W, ok[u], alpha ? key[u] : Y, alpha ? Y : key[u], hk[u], H[u], cw[u]);
}

// Singles: lane = single s of the column (alpha entries first); the value is
// h_ia plus the terms of the occupied spin-orbitals in spin-orbital order
// (W3 for the single's spin, V3 for the other), one running sum.
__device__ __forceinline__ void mc_item_s(const Problem &P, McWarp &W, const ColEnt *tA, int nsA, int ns, int s,
                                          unsigned long long A, unsigned long long B, unsigned long long hA,
                                          unsigned long long hB) {
    const int N = P.N;
    bool ok = false;
    unsigned long long oa = 0ull, ob = 0ull, hk = 0ull;
    double H = 0.0;
    unsigned cw = 0u;
    if (s < ns) {
        const ColEnt e = tA[s];
        const bool alpha = s < nsA;
        const int i = (e.info >> 8) & 0xff, a = (e.info >> 16) & 0xff;
        const size_t row = (size_t)(i * N + a) * N;
        const double *tA_row = (alpha ? P.W3 : P.V3) + row, *tB_row = (alpha ? P.V3 : P.W3) + row;
        double v = __ldg(P.h + i * N + a);
        for (unsigned long long m = A; m; m &= m - 1) v += __ldg(tA_row + (__ffsll((long long)m) - 1));
        for (unsigned long long m = B; m; m &= m - 1) v += __ldg(tB_row + (__ffsll((long long)m) - 1));
        H = apply_parity(v, (unsigned long long)(e.info & 1));
        oa = alpha ? e.key : A;
        ob = alpha ? B : e.key;
        hk = alpha ? (e.h ^ hB) : (hA ^ e.h);
        cw = cnz_word(P, hk, W.pol_last);
        ok = true;
    }
    mc_push(W, ok, oa, ob, hk, H, cw);
}

__global__ void __launch_bounds__(256, 3) k_mc_scatter(Problem P, McState *ms, IterState *st, const McSel *sel,
                                                    const ColEnt *coltab, const ColLists *collists, McGeom Gm,
                                                    const double *w, const double *thr, long long *cand,
                                                    double *gathp, unsigned int *work, McUpdate U) {
    __shared__ unsigned long long q_a[8][kScatterQ], q_b[8][kScatterQ], q_h[8][kScatterQ];
    __shared__ double q_H[8][kScatterQ];
    __shared__ long long w_cand[8][kWarpCand];
    __shared__ int s_cnt[4][8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (ms->done || st->status) return;
    const int m = ms->m_sel;
    if (U.on && blockIdx.x == 0) {                      // the first block: mu, alpha and the scale, beside the scatter
        mc_update_block(P, ms, st, U.cI, U.bI, U.eta, U.Rh, U.Rl, U.ldr, m, reinterpret_cast<float *>(&q_H[0][0]),
                        reinterpret_cast<double *>(&q_a[0][0]));
        return;
    }
    const int total = m * Gm.per_col;
    const int ns = Gm.nsA + Gm.nsB;
    McWarp W{q_a[warp], q_b[warp], q_h[warp], q_H[warp], w_cand[warp], l2_evict_first(), l2_evict_last(),
             0ull, 0.0, 0.0, 0, 0, 0, 0, 0, 0, false};
    // the next item's index is fetched while the current one runs
    int t_next = 0;
    if (lane == 0) t_next = (int)atomicAdd(work, 1u);
    t_next = __shfl_sync(0xffffffffu, t_next, 0);
    for (;;) {
        const int t = t_next;
        if (t >= total || W.err) break;
        unsigned int fetched = 0u;
        if (lane == 0) fetched = atomicAdd(work, 1u);
        const int col = t / Gm.per_col, k = t - col * Gm.per_col;
        const McSel xs = sel[col];
        W.wi = w[col];
        W.tib = abs_bits(thr[col]);
        W.gather = 0.0;
        const ColEnt *tA = coltab + (size_t)col * ns;
        if (k < Gm.n_ab) {
            const int lg = k / Gm.ab_ch, ch = k - lg * Gm.ab_ch;
            mc_item_ab(P, W, tA, tA + Gm.nsA, Gm.nsB, 32 * lg + lane, ch * kAbChunk, min(Gm.nsA, (ch + 1) * kAbChunk));
        } else if (k < Gm.n_ab + Gm.n_aa + Gm.n_bb) {
            const bool alpha = k < Gm.n_ab + Gm.n_aa;
            const int kk = k - (alpha ? Gm.n_ab : Gm.n_ab + Gm.n_aa);
            const int chn = alpha ? Gm.aa_ch : Gm.bb_ch;
            const int lg = kk / chn, ch = kk - lg * chn;
            const int co2 = alpha ? P.ca2 : P.cb2;
            const unsigned long long X = alpha ? xs.A : xs.B, Y = alpha ? xs.B : xs.A;
            const unsigned long long hY = alpha ? hash_beta(xs.B) : hash_alpha(xs.A);
            mc_item_ss(P, W, alpha, X, Y, hY, collists[col], 32 * lg + lane, ch * kSsChunk,
                       min(co2, (ch + 1) * kSsChunk));
        } else {
            const int lg = k - (Gm.n_ab + Gm.n_aa + Gm.n_bb);
            mc_item_s(P, W, tA, Gm.nsA, ns, 32 * lg + lane, xs.A, xs.B, hash_alpha(xs.A), hash_beta(xs.B));
        }
        mc_drain(P, ms, st, cand, W);
        // the item's gather: a fixed tree over the warp
        double gsum = W.gather;
        for (int o = 16; o > 0; o >>= 1) gsum += __shfl_down_sync(0xffffffffu, gsum, o);
        if (lane == 0) gathp[(size_t)col * Gm.per_col + k] = gsum;
        t_next = __shfl_sync(0xffffffffu, (int)fetched, 0);
    }
    mc_flush_cand(P, ms, st, w_cand[warp], W.nwc, cand);
    // counters: warp sums, then the warps in order
    const int r0 = __reduce_add_sync(0xffffffffu, W.c_el), r1 = __reduce_add_sync(0xffffffffu, W.c_app);
    const int r2 = __reduce_add_sync(0xffffffffu, W.c_drop), r3 = __reduce_add_sync(0xffffffffu, W.c_ins);
    if (lane == 0) { s_cnt[0][warp] = r0; s_cnt[1][warp] = r1; s_cnt[2][warp] = r2; s_cnt[3][warp] = r3; }
    __syncthreads();
    if (tid < 4) {
        unsigned long long t = 0;
        for (int q = 0; q < 8; ++q) t += (unsigned long long)s_cnt[tid][q];
        atomicAdd((unsigned long long *)&ms->cnt[tid], t);
    }
}

// b_I recalculated (Eq. recalculate-b), the chosen coordinates join the
// candidates, counters and the host snapshot.  One warp per chosen column (8
// per block): its gather from the item partials (lane-strided in item order,
// then a fixed tree), b_i = H_ii c_i + gather, the candidate mark; the block's
// new candidates in one reservation.  The last block to finish (a counter in
// McState, reset by that block) writes the counters and the snapshot.
constexpr int kFinWarps = 8;
__global__ void __launch_bounds__(32 * kFinWarps) k_mc_finalize(Problem P, McState *ms, IterState *st,
                                                                const McSel *sel, const double *Hdiag,
                                                                const double *gathp, long long *cand,
                                                                const double *etaout, int per_col, unsigned int *work) {
    __shared__ long long s_slot[kFinWarps];
    __shared__ int s_app[kFinWarps], s_nd[kFinWarps];
    __shared__ bool s_last;
    if (blockIdx.x == 0 && threadIdx.x == 0) *work = 0u;   // the next scatter's item counter
    if (ms->done) return;                               // read-only here: uniform over the blocks
    const bool skip = st->status != 0;
    const int m = ms->m_sel;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * kFinWarps + warp;
    if (lane == 0) { s_app[warp] = 0; s_nd[warp] = 0; }
    if (!skip && i < m) {                               // warp-uniform
        double t = 0.0;
        for (int k = lane; k < per_col; k += 32) t += gathp[(size_t)i * per_col + k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) {
            const long long slot = sel[i].slot;
            const double hd = Hdiag[i];
            Slot *sp = P.table + slot;
            sp->bv = fma(hd, sp->c, t);
            s_nd[warp] = is_zero(hd) ? 0 : 1;
            s_slot[warp] = slot;
            s_app[warp] = mark_set(P, slot) ? 1 : 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // the block's new candidates (warp order) in one reservation, its nonzero diagonals
        int na = 0, nd = 0;
        for (int w = 0; w < kFinWarps; ++w) { na += s_app[w]; nd += s_nd[w]; }
        if (na) {
            const int base = atomicAdd(&ms->n_cand, na);
            for (int w = 0, at = base; w < kFinWarps; ++w)
                if (s_app[w]) {
                    if (at < P.cap_cand) cand[at] = s_slot[w];
                    else set_status(st, kErrInternal);
                    ++at;
                }
        }
        if (nd) atomicAdd(&ms->fin_nd, nd);
        __threadfence();
        s_last = atomicAdd(&ms->fin_blocks, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    // every field read first (independent loads), then written
    const long long nd_all = (long long)atomicExch(&ms->fin_nd, 0);
    ms->fin_blocks = 0u;
    const unsigned long long c0 = ms->cnt[0], c1 = ms->cnt[1], c2 = ms->cnt[2], c3 = ms->cnt[3];
    const long long el = ms->elements + (long long)c0 + nd_all, ap = ms->applied + (long long)c1 + nd_all;
    const long long dr = ms->dropped + (long long)c2, in = ms->inserted + (long long)c3;
    const long long ns = ms->n_slots + (long long)c3;
    const long long its = ms->iterations, nnz = ms->nnz_c, eit = ms->eig_iters_total;
    const dd mu = ms->mu, al = ms->alpha;
    const double dx = ms->dx, en = ms->energy;
    const int done = ms->done_pending ? 1 : ms->done;
    const double eta0 = m > 0 ? etaout[0] : 0.0;
    const unsigned long long la = m > 0 ? sel[0].A : 0ull, lb = m > 0 ? sel[0].B : 0ull;
    ms->elements = el;
    ms->applied = ap;
    ms->dropped = dr;
    ms->inserted = in;
    ms->n_slots = ns;
    ms->last_column = (long long)c0 + nd_all;
    for (int k = 0; k < 4; ++k) ms->cnt[k] = 0;
    ms->done = done;
    if (ns > P.max_entries) set_status(st, kErrTableFull);
    st->iterations = its;
    st->nnz_c = nnz;
    st->n_slots = ns;
    st->elements = el;
    st->applied = ap;
    st->dropped = dr;
    st->inserted = in;
    st->last_column = (long long)c0 + nd_all;
    st->eig_iters = eit;
    st->mu = mu;
    st->alpha = al;
    st->dx = dx;
    st->energy = en;
    st->last_eta = eta0;
    st->last_a = la;
    st->last_b = lb;
    st->done = done;
}

// One entry of a start vector: c_{A,B} = eta from c = 0, as a forced block step
// of one coordinate (its column is scattered with weight eta by k_mc_scatter,
// b_{A,B} recalculated by k_mc_finalize).  mu += eta^2, alpha += 2 eta b + eta^2
// H (double-double), b as stored before the step.  The first entry (first = 1)
// starts from the reset state: c = e_ref (eta = 1) is the default start of r4.
__global__ void k_mc_start(Problem P, McState *ms, IterState *st, McSel *sel, double *Hdiag, double *w, double *thr,
                           double *etaout, unsigned long long A, unsigned long long B, double eta, int first,
                           ColEnt *coltab, ColLists *collists) {
    __shared__ ColLists L;
    __shared__ long long s_slot;
    __shared__ double s_bold;
    __shared__ int s_ins;
    if (threadIdx.x == 0) {
        bool ins = false;
        long long s = table_find(P, st, A, B, true, &ins);
        if (s < 0) { set_status(st, kErrTableFull); s = 0; }
        s_slot = s;
        s_ins = ins ? 1 : 0;
        s_bold = P.table[s].bv;
        P.table[s].c = eta;
        cnz_set(P, A, B);
    }
    for (int t = threadIdx.x; t < P.N; t += blockDim.x) {
        int ra = __popcll(A & low_mask(t)), rb = __popcll(B & low_mask(t));
        if ((A >> t) & 1ull) L.occA[ra] = (unsigned char)t; else L.virA[t - ra] = (unsigned char)t;
        if ((B >> t) & 1ull) L.occB[rb] = (unsigned char)t; else L.virB[t - rb] = (unsigned char)t;
    }
    __syncthreads();
    // the column's single excitations and orbital lists for the scatter (column 0)
    mc_build_coltab(P, L, A, B, coltab, threadIdx.x, blockDim.x);
    if (threadIdx.x < 32) reinterpret_cast<uint2 *>(collists)[threadIdx.x] = reinterpret_cast<const uint2 *>(&L)[threadIdx.x];
    if (threadIdx.x < 32) {
        const double hd = diag_warp(P, L);
        if (threadIdx.x == 0) {
            if (first) {
                ms->n_cand = 0;
                ms->mu = dd_from(0.0);
                ms->alpha = dd_from(0.0);
                ms->scale = dd_from(1.0);
                st->scale = dd_from(1.0);
                ms->dx = 0.0;
                ms->iterations = 0;
                ms->nnz_c = 0;
                ms->n_slots = 0;
                ms->inserted = 0;
                ms->elements = 0; ms->applied = 0; ms->dropped = 0; ms->last_column = 0;
                for (int k = 0; k < 4; ++k) ms->cnt[k] = 0;
                ms->done = 0;
                ms->done_pending = 0;
                ms->n_above = 0;
                ms->n_inbin = 0;
            }
            McSel x;
            x.slot = s_slot; x.gkey = 0ull; x.A = A; x.B = B;
            sel[0] = x;
            Hdiag[0] = hd;
            w[0] = eta;
            thr[0] = eta != 0.0 ? P.tau / fabs(eta) : 1.0e308;
            etaout[0] = eta;
            ms->m_sel = 1;
            ms->mu = dd_add(ms->mu, dd_two_prod(eta, eta));
            ms->alpha = dd_add(ms->alpha, dd_add(dd_two_prod(2.0 * eta, s_bold), dd_mul_d(dd_two_prod(eta, eta), hd)));
            ms->energy = ms->mu.hi != 0.0 ? dd_div_to_d(ms->alpha, ms->mu) : 0.0;
            ms->nnz_c += eta != 0.0 ? 1 : 0;
            ms->n_slots += s_ins;
            ms->inserted += s_ins;
        }
    }
}

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
size_t mc_eigen_smem(int m) {
    const int n1 = m + 1;
    const EigCfg g = eig_cfg(n1);
    size_t r;
    if (g.C == 1) r = 2 * (size_t)n1 * (size_t)eig_ldr(n1);          // R in one CTA
    else if (g.C > 1) r = 2 * (size_t)g.crows * (size_t)eig_ldr(n1);  // this CTA's rows of R
    else r = 2 * (size_t)eig_len(n1) + 4 * (size_t)eig_stage_rows(n1) * eig_ldr(n1);   // streamed
    return (r + eig_vec_floats(n1)) * sizeof(float);
}
int mc_eigen_threads(int m) {
    const EigCfg g = eig_cfg(m + 1);
    return g.tpr * 32 * ((g.crows + 31) / 32);
}
int mc_eigen_cluster(int m) { return eig_cfg(m + 1).C; }
int mc_ldr(int m) { return eig_ldr(m + 1); }
int mc_max_m() { return kEigMaxN - 1; }

// the scatter's grid: the blocks that are resident at once on this device (warps take items from a counter)
int mc_scatter_grid(const Problem &P) {
    (void)P;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mc_scatter, 256, 0) != cudaSuccess)
        return 0;
    return sms * std::max(per, 1);
}
// the scatter's work items per column (see k_mc_scatter)
McGeom mc_geometry(const Problem &P) {
    McGeom g{};
    g.nsA = P.na * P.va;
    g.nsB = P.nb * P.vb;
    if (!P.doubles_vanish) {
        g.ab_ch = (g.nsA + kAbChunk - 1) / kAbChunk;
        g.n_ab = g.nsB > 0 ? ((g.nsB + 31) / 32) * g.ab_ch : 0;
        g.aa_ch = (P.ca2 + kSsChunk - 1) / kSsChunk;
        g.n_aa = P.cva2 > 0 ? ((P.cva2 + 31) / 32) * g.aa_ch : 0;
        g.bb_ch = (P.cb2 + kSsChunk - 1) / kSsChunk;
        g.n_bb = P.cvb2 > 0 ? ((P.cvb2 + 31) / 32) * g.bb_ch : 0;
    }
    g.n_s = (g.nsA + g.nsB + 31) / 32;
    g.per_col = g.n_ab + g.n_aa + g.n_bb + g.n_s;
    return g;
}

cudaError_t mc_configure() {
    size_t most1 = 0, most0 = 0, most_cl = 0;
    for (int m = 1; m < kEigMaxN; ++m) {
        const int C = eig_cfg(m + 1).C;
        size_t &t = C > 1 ? most_cl : (C == 1 ? most1 : most0);
        t = std::max(t, mc_eigen_smem(m));
    }
    cudaError_t e = cudaFuncSetAttribute(k_mc_eigen<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)most1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_mc_eigen<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most0);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_mc_eigen<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most_cl);
    if (e != cudaSuccess) return e;
    return cudaSuccess;
}

// One matrix element H_{D'D} (Eq. entry; the get_entry / get_diagonal of Sec. "The Hamiltonian Class"):
// the diagonal by diag_warp, any other pair by hij_pair (zero beyond a double excitation).  One warp.
__global__ void k_entry(Problem P, unsigned long long A1, unsigned long long B1, unsigned long long A2,
                        unsigned long long B2, double *out) {
    __shared__ ColLists L;
    const int lane = threadIdx.x & 31;
    if (A1 == A2 && B1 == B2) {
        for (int t = lane; t < P.N; t += 32) {
            int ra = __popcll(A2 & low_mask(t)), rb = __popcll(B2 & low_mask(t));
            if ((A2 >> t) & 1ull) L.occA[ra] = (unsigned char)t; else L.virA[t - ra] = (unsigned char)t;
            if ((B2 >> t) & 1ull) L.occB[rb] = (unsigned char)t; else L.virB[t - rb] = (unsigned char)t;
        }
        __syncwarp();
        const double d = diag_warp(P, L);
        if (lane == 0) *out = d;
    } else if (lane == 0) {
        *out = hij_pair(P, A1, B1, A2, B2);
    }
}

cudaError_t launch_entry(const Problem &P, unsigned long long A1, unsigned long long B1, unsigned long long A2,
                         unsigned long long B2, double *out, cudaStream_t s) {
    k_entry<<<1, 32, 0, s>>>(P, A1, B1, A2, B2, out);
    return cudaGetLastError();
}

cudaError_t launch_mc_start(const Problem &P, const McBuffers &b, unsigned long long A, unsigned long long B,
                            double eta, int first, cudaStream_t s) {
    k_mc_start<<<1, 64, 0, s>>>(P, b.ms, b.st, b.sel, b.Hdiag, b.w, b.thr, b.eta, A, B, eta, first, b.coltab,
                                b.collists);
    return cudaGetLastError();
}

cudaError_t launch_mc_scatter_finalize(const Problem &P, const McBuffers &b, cudaStream_t s) {
    k_mc_scatter<<<b.scatter_grid, 256, 0, s>>>(P, b.ms, b.st, b.sel, b.coltab, b.collists, b.geom, b.w, b.thr,
                                                 b.cand, b.gathp, b.work, McUpdate{});
    k_mc_finalize<<<(b.m + kFinWarps - 1) / kFinWarps, 32 * kFinWarps, 0, s>>>(P, b.ms, b.st, b.sel, b.Hdiag, b.gathp,
                                                                              b.cand, b.eta, b.geom.per_col, b.work);
    return cudaGetLastError();
}

cudaError_t launch_mc_iteration(const Problem &P, const McBuffers &b, cudaStream_t s, cudaEvent_t *ev) {
    // ev (optional): kMcKernels + 1 events, recorded before every launch and after the last
    int k = 0;
    auto mark = [&]() {
        if (ev) cudaEventRecord(ev[k], s);
        ++k;
    };
    mark();
    k_mc_gkeys<<<b.cand_grid, 256, 0, s>>>(P, b.ms, b.st, b.cand, b.gkey, b.hist, b.m);
    mark();
    k_mc_hist<<<(b.cand_grid + 3) / 4, kHistThreads, 0, s>>>(b.ms, b.gkey, b.hist, b.cap_cand);
    mark();
    k_mc_collect<<<b.cand_grid, 256, 0, s>>>(P, b.ms, b.cand, b.gkey, b.sel, b.inbin);
    mark();
    k_mc_sortsel<<<1, 1024, 0, s>>>(P, b.ms, b.sel, b.inbin, b.m, b.st, b.cand, b.gkey, b.ties);
    mark();
    k_mc_prepare<<<(b.m + kPrepWarps - 1) / kPrepWarps, 32 * kPrepWarps, 0, s>>>(
        P, b.ms, b.sel, b.cI, b.bI, b.Hdiag, b.HIIc, b.rowf, b.Rh, b.Rl, b.ldr, b.coltab, b.collists,
        b.geom.nsA + b.geom.nsB);
    mark();
    {
        const EigCfg g = eig_cfg(b.m + 1);
        if (g.C > 1) {                                  // a cluster holding R's rows
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)g.C);
            cfg.blockDim = dim3((unsigned)mc_eigen_threads(b.m));
            cfg.dynamicSmemBytes = mc_eigen_smem(b.m);
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = (unsigned)g.C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            cudaLaunchKernelEx(&cfg, k_mc_eigen<true, true>, P, b.ms, b.st, (const McSel *)b.sel,
                               (const double *)b.cI, (const double *)b.bI, (const double *)b.HIIc,
                               (const double *)b.Hdiag, (const float4 *)b.rowf, b.Rh, b.Rl, b.ldr, g.tpr, g.crows,
                               b.w, b.thr, b.eta);
        } else if (g.C == 1) {                          // one CTA, R in its shared memory
            k_mc_eigen<false, true><<<1, mc_eigen_threads(b.m), mc_eigen_smem(b.m), s>>>(
                P, b.ms, b.st, b.sel, b.cI, b.bI, b.HIIc, b.Hdiag, b.rowf, b.Rh, b.Rl, b.ldr, g.tpr, b.m + 1, b.w,
                b.thr, b.eta);
        } else {                                        // one CTA streaming R from L2
            k_mc_eigen<false, false><<<1, mc_eigen_threads(b.m), mc_eigen_smem(b.m), s>>>(
                P, b.ms, b.st, b.sel, b.cI, b.bI, b.HIIc, b.Hdiag, b.rowf, b.Rh, b.Rl, b.ldr, g.tpr, b.m + 1, b.w,
                b.thr, b.eta);
        }
    }
    mark();
    // one more block than the scatter's own: block 0 updates mu, alpha and the scale meanwhile
    k_mc_scatter<<<b.scatter_grid + 1, 256, 0, s>>>(P, b.ms, b.st, b.sel, b.coltab, b.collists, b.geom, b.w, b.thr,
                                                     b.cand, b.gathp, b.work,
                                                     McUpdate{b.cI, b.bI, b.eta, b.Rh, b.Rl, b.ldr, 1});
    mark();
    k_mc_finalize<<<(b.m + kFinWarps - 1) / kFinWarps, 32 * kFinWarps, 0, s>>>(P, b.ms, b.st, b.sel, b.Hdiag, b.gathp,
                                                                              b.cand, b.eta, b.geom.per_col, b.work);
    mark();
    return cudaGetLastError();
}

}  // namespace cdfci
