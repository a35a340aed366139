// xCDFCI (Algorithm 3): K + 1 states, one row of C per iteration.
//
// Per iteration four launches (captured in a CUDA graph):
//   k_x_select    argmax over the candidates of ||G_j||_inf, G_j = 4 B_j + 4 C_j S
//                 (ties: the smaller key), by a block argmax and a last-block
//                 reduction in block order; clears the candidates' marks;
//   k_x_prepare   H_ii, the quartic of problem choose-eta (appendix "Determining
//                 Step Size") and its minimiser eta, C_i += eta G_i, the S and M
//                 updates (double-double, one entry per lane);
//   k_x_scatter   B_j += eta H_ji G_i for the column of i with the row compression
//                 rule, insertion of absent rows, the gather sum_j H_ji C_j per
//                 block, the rows it updated become the next candidates;
//   k_x_finalize  B_i = H_ii C_i + the gather (Eq. recalculate-b, per state),
//                 counters.
// The energies (the pencil (M, S)) are computed on request by k_x_energies.
// Each row j occurs once in a column, so B_j is updated by plain loads and
// stores, and every reduction has a fixed order: the iteration is
// deterministic.
#include <cooperative_groups.h>

#include <algorithm>

#include "cdfci_internal.cuh"
#include "cdfci_kernels.h"

namespace cdfci {

namespace cg = cooperative_groups;

namespace {

struct XBest {
    unsigned long long gbits, a, b;
    long long slot;
};

// |x| as its bit pattern (monotone in |x| for non-negative doubles)
__device__ __forceinline__ unsigned long long x_abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ bool x_better(const XBest &x, const XBest &y) {
    if (x.slot < 0) return false;
    if (y.slot < 0) return true;
    return x.gbits > y.gbits || (x.gbits == y.gbits && key_less(x.a, x.b, y.a, y.b));
}


// ||G_j||_inf and G_j = 4 B_j + 4 C_j S from the row's C and B halves (G may be null)
__device__ __forceinline__ double x_gnorm(const double (&c)[kXMax], const double (&bb)[kXMax], const double *S, int k1,
                                           double *G) {
    double m = 0.0;
#pragma unroll
    for (int a = 0; a < kXMax; ++a) {
        if (a >= k1) break;
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < kXMax; ++b) {
            if (b >= k1) break;
            s = fma(c[b], S[b * k1 + a], s);
        }
        const double ga = 4.0 * bb[a] + 4.0 * s;
        if (G) G[a] = ga;
        m = fmax(m, fabs(ga));
    }
    return m;
}

}  // namespace

constexpr int kXThreads = 256;

// Row j of C and of B (k1 values each) into cv and bv, all loads in flight
// together: 16-byte loads when k1 is even (each half is then whole pairs, and
// a row starts at a multiple of 16 bytes), else 8-byte ones.  The scatter is
// bound by the number of memory requests its elements make at once.
__device__ __forceinline__ void x_ld32(const double *p, double &a, double &b, double &c, double &d) {
    asm volatile("ld.global.cg.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a), "=d"(b), "=d"(c), "=d"(d) : "l"(p));
}
__device__ __forceinline__ void x_load_row(const double *rows, long long j, int k1, double (&cv)[kXMax],
                                           double (&bv)[kXMax]) {
    const double *r = rows + j * 2 * k1;
    if ((k1 & 3) == 0) {                                             // uniform: 32-byte loads (halves 32-byte aligned)
#pragma unroll
        for (int q = 0; q < kXMax / 4; ++q) {
            double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
            if (4 * q < k1) {
                x_ld32(r + 4 * q, c0, c1, c2, c3);
                x_ld32(r + k1 + 4 * q, b0, b1, b2, b3);
            }
            cv[4 * q] = c0; cv[4 * q + 1] = c1; cv[4 * q + 2] = c2; cv[4 * q + 3] = c3;
            bv[4 * q] = b0; bv[4 * q + 1] = b1; bv[4 * q + 2] = b2; bv[4 * q + 3] = b3;
        }
        return;
    }
    if ((k1 & 1) == 0) {                                             // uniform
        const double2 *r2 = reinterpret_cast<const double2 *>(r);
#pragma unroll
        for (int q = 0; q < kXMax / 2; ++q) {
            double2 c2 = make_double2(0.0, 0.0), b2 = c2;
            if (2 * q < k1) {
                c2 = __ldcg(r2 + q);
                b2 = __ldcg(r2 + k1 / 2 + q);
            }
            cv[2 * q] = c2.x; cv[2 * q + 1] = c2.y;
            bv[2 * q] = b2.x; bv[2 * q + 1] = b2.y;
        }
        return;
    }
#pragma unroll
    for (int a = 0; a < kXMax; ++a) {
        cv[a] = a < k1 ? __ldcg(r + a) : 0.0;
        bv[a] = a < k1 ? __ldcg(r + k1 + a) : 0.0;
    }
}

__global__ void __launch_bounds__(kXThreads) k_x_select(Problem P, XState *xs, IterState *st, const long long *cand,
                                                        const double *rows, XBest *bbest, unsigned int *counter) {
    __shared__ double sS[kXMax * kXMax];
    __shared__ XBest wb[kXThreads / 32];
    __shared__ bool s_last;
    if (xs->done || st->status) return;
    const int k1 = xs->k1, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < k1 * k1; t += blockDim.x) sS[t] = xs->S[t].hi + xs->S[t].lo;
    __syncthreads();
    const int n = xs->n_cand;
    XBest best{0ull, ~0ull, ~0ull, -1};
    for (int t = blockIdx.x * blockDim.x + tid; t < n; t += gridDim.x * blockDim.x) {
        const long long s = cand[t];
        double rc[kXMax], rb[kXMax];
        x_load_row(rows, s, k1, rc, rb);
        const ulonglong2 key = __ldcg(reinterpret_cast<const ulonglong2 *>(P.table + s));
        P.table[s].b = key.y & kKeyMaskB;                          // no longer a candidate
        const XBest x{x_abs_bits(x_gnorm(rc, rb, sS, k1, nullptr)), key.x, key.y & kKeyMaskB, s};
        if (x_better(x, best)) best = x;
    }
    for (int off = 16; off > 0; off >>= 1) {
        XBest y;
        y.gbits = __shfl_down_sync(0xffffffffu, best.gbits, off);
        y.a = __shfl_down_sync(0xffffffffu, best.a, off);
        y.b = __shfl_down_sync(0xffffffffu, best.b, off);
        y.slot = __shfl_down_sync(0xffffffffu, best.slot, off);
        if (x_better(y, best)) best = y;
    }
    if (lane == 0) wb[warp] = best;
    __syncthreads();
    if (tid == 0) {
        XBest b = wb[0];
        for (int w = 1; w < kXThreads / 32; ++w)
            if (x_better(wb[w], b)) b = wb[w];
        bbest[blockIdx.x] = b;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || warp != 0) return;
    __threadfence();
    // the last block's warp 0 reduces the blocks' winners: lane l takes blocks l, l + 32, ...
    XBest b{0ull, ~0ull, ~0ull, -1};
    for (int k = lane; k < (int)gridDim.x; k += 32) {
        const XBest y = bbest[k];
        if (x_better(y, b)) b = y;
    }
    for (int off = 16; off > 0; off >>= 1) {
        XBest y;
        y.gbits = __shfl_down_sync(0xffffffffu, b.gbits, off);
        y.a = __shfl_down_sync(0xffffffffu, b.a, off);
        y.b = __shfl_down_sync(0xffffffffu, b.b, off);
        y.slot = __shfl_down_sync(0xffffffffu, b.slot, off);
        if (x_better(y, b)) b = y;
    }
    if (lane != 0) return;
    *counter = 0u;
    xs->n_cand = 0;
    if (b.slot < 0) { xs->done = 1; xs->eta = 0.0; return; }     // nothing left to choose
    double rc[kXMax], rb[kXMax], G[kXMax];
    x_load_row(rows, b.slot, k1, rc, rb);
    x_gnorm(rc, rb, sS, k1, G);
    for (int a = 0; a < k1; ++a) xs->g[a] = G[a];
    xs->slot = b.slot; xs->A = b.a; xs->B = b.b;
}

// H_ii exactly as diag_warp(P, L) computes it (the same terms, per-lane sums
// in the same order, the same tree), with every lane's loads issued before the
// first addition: one round trip for the integrals of up to 16 electrons.
__device__ __forceinline__ double x_diag(const Problem &P, const ColLists &L) {
    const int lane = threadIdx.x & 31;
    const int N = P.N, n = P.na + P.nb, n2 = n * n;
    if (n > 16) return diag_warp(P, L);                               // more than two rounds per lane
    const int ph = lane < n ? (lane < P.na ? L.occA[lane] : L.occB[lane - P.na]) : 0;
    const double hv = lane < n ? __ldg(P.h + ph * (N + 1)) : 0.0;
    double tv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {                                     // t = lane + 128 (k / 4) + 32 (k % 4)
        const int t = lane + 128 * (k >> 2) + 32 * (k & 3);
        tv[k] = 0.0;
        if (t < n2) {
            const int u = t / n, w = t - u * n;
            if (u != w) {
                const bool ua = u < P.na, wa = w < P.na;
                const int p = ua ? L.occA[u] : L.occB[u - P.na];
                const int q = wa ? L.occA[w] : L.occB[w - P.na];
                const double jv = P.J[p * N + q];
                tv[k] = (ua == wa) ? (jv - P.K[p * N + q]) : jv;
            }
        }
    }
    double x = 0.0;
    if (lane < n) x += hv;
    double y4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int t = lane + 128 * (k >> 2) + 32 * (k & 3);
        if (t < n2) {
            const int u = t / n, w = t - u * n;
            if (u != w) y4[k & 3] += tv[k];
        }
    }
    x = fma(0.5, (y4[0] + y4[1]) + (y4[2] + y4[3]), x);
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    return __shfl_sync(0xffffffffu, x, 0);
}

// forced >= 0: the start step of row {fA, fB} with g = e_forced and eta = 1.
__global__ void k_x_prepare(Problem P, XState *xs, IterState *st, double *rows, int forced, unsigned long long fA,
                            unsigned long long fB) {
    __shared__ ColLists L;
    __shared__ long long s_slot;
    __shared__ double s_c[kXMax], s_g[kXMax], s_b[kXMax], s_t[kXMax];
    __shared__ double s_eta, s_gn, s_w[kXMax];
    __shared__ int s_stop;
    if (xs->done || st->status) return;
    const int k1 = xs->k1, lane = threadIdx.x;
    if (lane == 0) {
        s_stop = 0;
        xs->eta = 0.0;                                               // 0: no step this iteration
        if (forced >= 0) {
            bool ins = false;
            const long long s = table_find(P, st, fA, fB, true, &ins);
            if (s < 0) { s_stop = 1; } else {
                if (ins) { xs->n_slots += 1; xs->inserted += 1; }
                xs->slot = s; xs->A = fA; xs->B = fB;
                for (int a = 0; a < k1; ++a) xs->g[a] = a == forced ? 1.0 : 0.0;
            }
        }
        s_slot = xs->slot;
    }
    __syncwarp();
    if (s_stop) return;
    build_lists(L, P.N, xs->A, xs->B);
    const long long s = s_slot;
    if (lane < k1) {                                                  // loads in flight beside H_ii's
        s_c[lane] = rows[s * 2 * k1 + lane];
        s_b[lane] = rows[s * 2 * k1 + k1 + lane];
        s_g[lane] = xs->g[lane];
    }
    __syncwarp();
    const double Hii = x_diag(P, L);
    if (lane < k1 && forced < 0) {                                    // (S g)_a, lane a: the term of g S g^T
        double t = 0.0;
        for (int b = 0; b < k1; ++b) t = fma(xs->S[lane * k1 + b].hi + xs->S[lane * k1 + b].lo, s_g[b], t);
        s_t[lane] = t;
    }
    __syncwarp();
    if (lane == 0) {
        double eta = 1.0;
        if (forced < 0) {
            // h(eta) = f(C + eta e_i g) - f(C) = w4 eta^4 + w3 eta^3 + w2 eta^2 + w1 eta with w4 = ||g||^4,
            // w3 = 4 ||g||^2 c.g, w2 = 2 H_ii ||g||^2 + 2 (c.g)^2 + 2 ||c||^2 ||g||^2 + 2 g S g^T,
            // w1 = ||g||^2 (the directional derivative)
            double gg = 0.0, cg = 0.0, cc = 0.0, gSg = 0.0;
            for (int a = 0; a < k1; ++a) {
                gg = fma(s_g[a], s_g[a], gg);
                cg = fma(s_c[a], s_g[a], cg);
                cc = fma(s_c[a], s_c[a], cc);
                gSg = fma(s_g[a], s_t[a], gSg);
            }
            // In t = eta ||g|| the quartic is monic with O(1) coefficients (w / w4 would grow like
            // 1 / ||g||^2 near convergence and overflow the single-precision root stage):
            // t^4 + 4 (c.u) t^3 + (2 H_ii + 2 (c.u)^2 + 2 ||c||^2 + 2 u S u^T) t^2 + ||g|| t, u = g / ||g||.
            const double gn = sqrt(gg);
            s_gn = gn;
            if (!(gn > 0.0)) { xs->done = 1; s_stop = 1; }
            else {
                const double cu = cg / gn;
                const double v3 = 4.0 * cu;
                const double v2 = 2.0 * Hii + 2.0 * cu * cu + 2.0 * cc + 2.0 * (gSg / gg);
                eta = line_search(gn, v2, v3) / gn;
                if (!isfinite(eta)) { set_status(st, kErrNonfinite); s_stop = 1; }
            }
        }
        s_eta = eta;
    }
    __syncwarp();
    if (s_stop) return;
    const double eta = s_eta;
    // S += eta (c^T g + g^T c) + eta^2 g^T g,  M += eta (b^T g + g^T b) + eta^2 H_ii g^T g (one entry per lane)
    for (int t = lane; t < k1 * k1; t += 32) {
        const int a = t / k1, b = t - a * k1;
        const dd e2 = dd_two_prod(eta, eta);
        const dd gab = dd_two_prod(s_g[a], s_g[b]);
        const dd ds = dd_add(dd_mul_d(dd_add(dd_two_prod(s_c[a], s_g[b]), dd_two_prod(s_g[a], s_c[b])), eta),
                             dd_mul(e2, gab));
        const dd dm = dd_add(dd_mul_d(dd_add(dd_two_prod(s_b[a], s_g[b]), dd_two_prod(s_g[a], s_b[b])), eta),
                             dd_mul_d(dd_mul(e2, gab), Hii));
        xs->S[t] = dd_add(xs->S[t], ds);
        xs->M[t] = dd_add(xs->M[t], dm);
    }
    // C_i += eta g (lane a), the scatter weights eta g and their largest magnitude
    const bool on = lane < k1;
    double cn = 0.0;
    if (on) {
        cn = fma(eta, s_g[lane], s_c[lane]);
        rows[s * 2 * k1 + lane] = cn;
        const double wa = eta * s_g[lane];
        xs->wv[lane] = wa;
        s_w[lane] = fabs(wa);
    }
    const unsigned was = __ballot_sync(0xffffffffu, on && s_c[lane] != 0.0);
    const unsigned now = __ballot_sync(0xffffffffu, on && cn != 0.0);
    __syncwarp();
    if (lane == 0) {
        double wmax = 0.0;
        for (int a = 0; a < k1; ++a) wmax = fmax(wmax, s_w[a]);
        xs->nnz_c += (now ? 1 : 0) - (was ? 1 : 0);
        xs->thr = wmax > 0.0 ? P.tau / wmax : 1.0e308;
        xs->eta = eta;
        xs->Hii = Hii;
        if (forced < 0) {
            xs->dx = P.theta * xs->dx + (1.0 - P.theta) * fabs(eta) * s_gn;   // s_gn = ||g||
            xs->iterations += 1;
            if (P.dx_threshold > 0.0 && xs->dx < P.dx_threshold) xs->done = 1;
        }
    }
}


// The slot of key {a, b} by linear probing from pos (no insert): -1 absent, -2
// error (status set); kbo receives the slot's b word, candidate mark included.
__device__ __forceinline__ long long x_find(const Problem &P, IterState *st, unsigned long long a,
                                            unsigned long long b, unsigned long long pos, unsigned long long &kbo) {
    const bool both_nonzero = (P.na > 0) && (P.nb > 0);
    for (int probe = 0; probe < P.max_probe; ++probe) {
        const Slot *s = P.table + pos;
        ulonglong2 k = __ldcg(reinterpret_cast<const ulonglong2 *>(s));         // the key in one request
        int spins = 0;
        while (both_nonzero && ((k.x == 0ull) != (k.y == 0ull))) {   // an insert in flight
            if (++spins > (1 << 20)) { set_status(st, kErrTimeout); return -2; }
            k = __ldcg(reinterpret_cast<const ulonglong2 *>(s));
        }
        const unsigned long long ka = k.x, kb = k.y;
        if (ka == a && (kb & kKeyMaskB) == b) { kbo = kb; return (long long)pos; }
        if (ka == 0ull && kb == 0ull) return -1;
        pos = (pos + 1) & P.mask;
    }
    set_status(st, kErrTableFull);
    return -2;
}

__global__ void __launch_bounds__(kXThreads) k_x_scatter(Problem P, XState *xs, IterState *st, double *rows,
                                                         long long *cand, long long cap_cand, double *gathp) {
    __shared__ ColLists L;
    __shared__ double sw[kXMax];
    __shared__ double sg[kXThreads / 32][kXMax];
    __shared__ unsigned int s_cnt[4][kXThreads / 32];
    if (xs->eta == 0.0 || st->status) return;                        // no step this iteration
    const int k1 = xs->k1, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long A = xs->A, B = xs->B;
    build_lists(L, P.N, A, B);
    if (tid < kXMax) sw[tid] = tid < k1 ? xs->wv[tid] : 0.0;
    __syncthreads();
    const double thr = xs->thr;
    const long long nh = P.doubles_vanish ? P.seg[2] : P.seg[5];
    double gat[kXMax];
#pragma unroll
    for (int a = 0; a < kXMax; ++a) gat[a] = 0.0;
    unsigned int c0 = 0, c1 = 0, c2 = 0, c3 = 0;                     // elements, applied, dropped, inserted
    for (long long e = 1 + (long long)blockIdx.x * blockDim.x + tid; e < nh; e += (long long)gridDim.x * blockDim.x) {
        unsigned long long oa, ob;
        const double H = column_element(P, L, A, B, e, oa, ob);
        if (is_zero(H)) continue;
        ++c0;
        // the row at the key's first probe position loads beside the key (it is usually found
        // there); no other thread of this launch writes row j or the mark of j (each row occurs
        // once in a column), so the values loaded here are current
        const unsigned long long pos0 = key_hash(oa, ob) & P.mask;
        double rc[kXMax], rb[kXMax];
        x_load_row(rows, (long long)pos0, k1, rc, rb);
        unsigned long long kb = 0ull;
        long long s = x_find(P, st, oa, ob, pos0, kb);
        if (s >= 0 && s != (long long)pos0) x_load_row(rows, s, k1, rc, rb);
        double cj[kXMax];
        bool cnz = false;
#pragma unroll
        for (int a = 0; a < kXMax; ++a) {
            cj[a] = s >= 0 && a < k1 ? rc[a] : 0.0;
            cnz = cnz || cj[a] != 0.0;
        }
        if (!cnz && !(fabs(H) >= thr)) { ++c2; continue; }
        if (s < 0) {
            bool ins = false;
            s = table_find(P, st, oa, ob, true, &ins);
            if (s < 0) continue;                                      // table full: status set
            if (ins) ++c3;
            x_load_row(rows, s, k1, rc, rb);
            kb = __ldcg(&P.table[s].b);
        }
        ++c1;
        double *br = rows + s * 2 * k1 + k1;
        double bn[kXMax];
#pragma unroll
        for (int a = 0; a < kXMax; ++a) {
            bn[a] = fma(H, sw[a], rb[a]);
            if (a < k1) gat[a] = fma(H, cj[a], gat[a]);
        }
        if ((k1 & 3) == 0) {                                          // 32-byte stores (see x_load_row)
#pragma unroll
            for (int q = 0; q < kXMax / 4; ++q)
                if (4 * q < k1)
                    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(br + 4 * q), "d"(bn[4 * q]),
                                 "d"(bn[4 * q + 1]), "d"(bn[4 * q + 2]), "d"(bn[4 * q + 3])
                                 : "memory");
        } else if ((k1 & 1) == 0) {                                   // 16-byte stores (see x_load_row)
#pragma unroll
            for (int q = 0; q < kXMax / 2; ++q)
                if (2 * q < k1) reinterpret_cast<double2 *>(br)[q] = make_double2(bn[2 * q], bn[2 * q + 1]);
        } else {
#pragma unroll
            for (int a = 0; a < kXMax; ++a)
                if (a < k1) br[a] = bn[a];
        }
        if (!(kb & kMarkB)) {
            P.table[s].b = kb | kMarkB;
            // one reservation for the lanes that get here together (a warp-aggregated append)
            const cg::coalesced_group grp = cg::coalesced_threads();
            int base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(&xs->n_cand, (int)grp.size());
            const int pos = grp.shfl(base, 0) + (int)grp.thread_rank();
            if (pos < cap_cand) cand[pos] = s;
            else set_status(st, kErrInternal);
        }
    }
    // gather: warp tree, then warps in order (fixed order)
#pragma unroll
    for (int a = 0; a < kXMax; ++a) {
        if (a >= k1) break;
        double v = gat[a];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sg[warp][a] = v;
    }
    // counters: warp sums (no shared-memory atomics), then the warps in order
    c0 = __reduce_add_sync(0xffffffffu, c0); c1 = __reduce_add_sync(0xffffffffu, c1);
    c2 = __reduce_add_sync(0xffffffffu, c2); c3 = __reduce_add_sync(0xffffffffu, c3);
    if (lane == 0) { s_cnt[0][warp] = c0; s_cnt[1][warp] = c1; s_cnt[2][warp] = c2; s_cnt[3][warp] = c3; }
    __syncthreads();
    if (tid < k1) {
        double v = sg[0][tid];
        for (int w = 1; w < kXThreads / 32; ++w) v += sg[w][tid];
        gathp[(size_t)blockIdx.x * k1 + tid] = v;
    }
    if (tid < 4) {
        unsigned long long t = 0;
        for (int w = 0; w < kXThreads / 32; ++w) t += s_cnt[tid][w];
        if (t) atomicAdd(&xs->cnt[tid], t);
    }
}

__global__ void __launch_bounds__(kXThreads) k_x_finalize(Problem P, XState *xs, IterState *st, double *rows,
                                                          const double *gathp, int nblocks, long long *cand,
                                                          long long cap_cand) {
    __shared__ double red[kXMax][kXThreads];
    if (xs->eta == 0.0 || st->status) return;                        // no step this iteration
    const int k1 = xs->k1, tid = threadIdx.x;
    const long long s = xs->slot;
    const double Hii = xs->Hii;
    // every state at once: per state, the thread's blocks in order, then the same pairwise tree
    double v[kXMax];
#pragma unroll
    for (int a = 0; a < kXMax; ++a) v[a] = 0.0;
    for (int k = tid; k < nblocks; k += blockDim.x) {
#pragma unroll
        for (int a = 0; a < kXMax; ++a)
            if (a < k1) v[a] += gathp[(size_t)k * k1 + a];
    }
#pragma unroll
    for (int a = 0; a < kXMax; ++a)
        if (a < k1) red[a][tid] = v[a];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (tid < w) {
#pragma unroll
            for (int a = 0; a < kXMax; ++a)
                if (a < k1) red[a][tid] += red[a][tid + w];
        }
        __syncthreads();
    }
    if (tid < k1) rows[s * 2 * k1 + k1 + tid] = fma(Hii, rows[s * 2 * k1 + tid], red[tid][0]);
    if (tid == 0) {
        const unsigned long long kb = P.table[s].b;
        if (!(kb & kMarkB)) {
            P.table[s].b = kb | kMarkB;
            const int pos = atomicAdd(&xs->n_cand, 1);
            if (pos < cap_cand) cand[pos] = s;
            else set_status(st, kErrInternal);
        }
        const long long nd = Hii != 0.0 ? 1 : 0;
        xs->elements += (long long)xs->cnt[0] + nd;
        xs->applied += (long long)xs->cnt[1] + nd;
        xs->dropped += (long long)xs->cnt[2];
        xs->inserted += (long long)xs->cnt[3];
        xs->n_slots += (long long)xs->cnt[3];
        xs->last_column = (long long)xs->cnt[0] + nd;
        for (int k = 0; k < 4; ++k) xs->cnt[k] = 0ull;
        if (xs->n_slots > P.max_entries) set_status(st, kErrTableFull);
    }
}

// Energies: the k1 eigenvalues of the pencil (M, S), ascending: S = L L^T
// (Cholesky), the symmetric A = L^-1 M L^-T, cyclic Jacobi rotations (Golub &
// Van Loan, Sec. 8.5) until the off-diagonal mass is below 1e-30 of the total.
// One thread; also the host-visible snapshot.
__global__ void k_x_energies(XState *xs, IterState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = xs->k1;
    double L[kXMax * kXMax], T[kXMax * kXMax], A[kXMax * kXMax];
    bool ok = true;
    for (int i = 0; i < n * n; ++i) L[i] = 0.0;
    for (int i = 0; i < n && ok; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = xs->S[i * n + j].hi + xs->S[i * n + j].lo;
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0.0)) { ok = false; break; }
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    if (ok) {
        for (int col = 0; col < n; ++col)
            for (int i = 0; i < n; ++i) {
                double s = xs->M[i * n + col].hi + xs->M[i * n + col].lo;
                for (int k = 0; k < i; ++k) s -= L[i * n + k] * T[k * n + col];
                T[i * n + col] = s / L[i * n + i];
            }
        for (int row = 0; row < n; ++row)
            for (int i = 0; i < n; ++i) {
                double s = T[row * n + i];
                for (int k = 0; k < i; ++k) s -= L[i * n + k] * A[row * n + k];
                A[row * n + i] = s / L[i * n + i];
            }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) {
                const double v = 0.5 * (A[i * n + j] + A[j * n + i]);
                A[i * n + j] = v; A[j * n + i] = v;
            }
        for (int sweep = 0; sweep < 64; ++sweep) {
            double off = 0.0, tot = 0.0;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    tot += A[i * n + j] * A[i * n + j];
                    if (i != j) off += A[i * n + j] * A[i * n + j];
                }
            if (off <= 1e-30 * tot) break;
            for (int p = 0; p < n; ++p)
                for (int q = p + 1; q < n; ++q) {
                    const double apq = A[p * n + q];
                    if (apq == 0.0) continue;
                    const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                    const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                    for (int k = 0; k < n; ++k) {
                        const double akp = A[k * n + p], akq = A[k * n + q];
                        A[k * n + p] = c * akp - sn * akq;
                        A[k * n + q] = sn * akp + c * akq;
                    }
                    for (int k = 0; k < n; ++k) {
                        const double apk = A[p * n + k], aqk = A[q * n + k];
                        A[p * n + k] = c * apk - sn * aqk;
                        A[q * n + k] = sn * apk + c * aqk;
                    }
                }
        }
        double E[kXMax];
        for (int i = 0; i < n; ++i) E[i] = A[i * n + i];
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j)
                if (E[j] < E[i]) { const double t = E[i]; E[i] = E[j]; E[j] = t; }
        for (int i = 0; i < n; ++i) xs->E[i] = E[i];
    } else {
        for (int i = 0; i < n; ++i) xs->E[i] = nan("");
    }
    st->iterations = xs->iterations; st->nnz_c = xs->nnz_c; st->n_slots = xs->n_slots;
    st->elements = xs->elements; st->applied = xs->applied; st->dropped = xs->dropped; st->inserted = xs->inserted;
    st->last_column = xs->last_column;
    st->mu = xs->S[0]; st->alpha = xs->M[0];
    st->dx = xs->dx; st->energy = xs->E[0]; st->last_eta = xs->eta;
    st->last_a = xs->A; st->last_b = xs->B; st->done = xs->done;
}

// Diagonal elements H_DD of a list of determinants (one warp each): picks the
// start rows of xCDFCI.
__global__ void k_x_diag_list(Problem P, const unsigned long long *keys, long long n, double *out) {
    __shared__ ColLists Ls[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ColLists &L = Ls[warp];
    for (long long k = (long long)blockIdx.x * 8 + warp; k < n; k += (long long)gridDim.x * 8) {
        const unsigned long long A = keys[2 * k], B = keys[2 * k + 1];
        for (int t = lane; t < P.N; t += 32) {
            const int ra = __popcll(A & low_mask(t)), rb = __popcll(B & low_mask(t));
            if ((A >> t) & 1ull) L.occA[ra] = (unsigned char)t; else L.virA[t - ra] = (unsigned char)t;
            if ((B >> t) & 1ull) L.occB[rb] = (unsigned char)t; else L.virB[t - rb] = (unsigned char)t;
        }
        __syncwarp();
        const double d = diag_warp(P, L);
        if (lane == 0) out[k] = d;
        __syncwarp();
    }
}

// Every stored determinant with its rows (k1 values of C and of B).
__global__ void k_x_export(Problem P, const double *rows, int k1, unsigned long long *keys, double *C, double *B,
                           long long cap, unsigned long long *counter) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.capacity;
         i += (long long)gridDim.x * blockDim.x) {
        const Slot sl = P.table[i];
        if (sl.a == 0ull && sl.b == 0ull) continue;
        const unsigned long long pos = atomicAdd(counter, 1ull);
        if ((long long)pos >= cap) continue;
        keys[2 * pos] = sl.a;
        keys[2 * pos + 1] = sl.b & kKeyMaskB;
        for (int a = 0; a < k1; ++a) {
            C[pos * k1 + a] = rows[i * 2 * k1 + a];
            B[pos * k1 + a] = rows[i * 2 * k1 + k1 + a];
        }
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
cudaError_t launch_x_export(const Problem &P, const XBuffers &b, int k1, unsigned long long *keys, double *C,
                            double *B, long long cap, unsigned long long *counter, cudaStream_t s) {
    long long grid = (P.capacity + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    k_x_export<<<(int)grid, 256, 0, s>>>(P, b.rows, k1, keys, C, B, cap, counter);
    return cudaGetLastError();
}

cudaError_t launch_x_diag_list(const Problem &P, const unsigned long long *keys, long long n, double *out,
                               cudaStream_t s) {
    const long long blocks = std::min<long long>((n + 7) / 8, 1024);
    k_x_diag_list<<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(P, keys, n, out);
    return cudaGetLastError();
}

int x_scatter_blocks() { return 152 * 2; }

size_t x_block_bytes() { return sizeof(XBest); }

cudaError_t launch_x_start(const Problem &P, const XBuffers &b, unsigned long long A, unsigned long long B, int k,
                           cudaStream_t s) {
    k_x_prepare<<<1, 32, 0, s>>>(P, b.xs, b.st, b.rows, k, A, B);
    k_x_scatter<<<b.nscatter, kXThreads, 0, s>>>(P, b.xs, b.st, b.rows, b.cand, b.cap_cand, b.gathp);
    k_x_finalize<<<1, kXThreads, 0, s>>>(P, b.xs, b.st, b.rows, b.gathp, b.nscatter, b.cand, b.cap_cand);
    return cudaGetLastError();
}

cudaError_t launch_x_iteration(const Problem &P, const XBuffers &b, cudaStream_t s) {
    k_x_select<<<b.nselect, kXThreads, 0, s>>>(P, b.xs, b.st, b.cand, b.rows, static_cast<XBest *>(b.bbest),
                                              b.counter);
    return launch_x_start(P, b, 0ull, 0ull, -1, s);
}

cudaError_t launch_x_energies(const XBuffers &b, cudaStream_t s) {
    k_x_energies<<<1, 32, 0, s>>>(b.xs, b.st);
    return cudaGetLastError();
}

}  // namespace cdfci
