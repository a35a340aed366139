// CUDA kernels of libcdfci (sm_103a).
//
// The m = 1 iteration (Algorithm 1) is one launch of k_cd_iter:
//   prologue  (every CTA, identical results): orbital lists of the chosen
//             determinant i, H_ii, the step size eta (appendix), the new
//             c_i, mu and alpha (Eq. update-var, double-double);
//   scatter   (grid-stride over the flat excitation index of column i): the
//             Slater-Condon element H_ji, the compression test
//             (c_j != 0 or |eta H_ji| >= tau), hash probe / 16-byte CAS
//             insert, atomicAdd of eta H_ji on b_j, the gather sum_j H_ji c_j
//             for the recalculation of b_i (Eq. recalculate-b), and the
//             running argmax of |4 b_j + 4 mu c_j| over the updated entries,
//             which are the candidates I_H(i) of the next choice (Eq. choose-i);
//   tail      (the last CTA to arrive): fixed-order reduction of the per-CTA
//             partials, the write of c_i and the recalculated b_i, the next
//             coordinate, the scalars and the counters.
// Within a column every j appears once, so atomicAdd returns the final b_j
// of this iteration and the fused argmax sees exactly the values the
// selection of Algorithm 1 would read.
#include "cdfci_internal.cuh"
#include "cdfci_kernels.h"

namespace cdfci {

__device__ __forceinline__ bool better(unsigned long long g1, unsigned long long a1, unsigned long long b1,
                                       unsigned long long g2, unsigned long long a2, unsigned long long b2) {
    return g1 > g2 || (g1 == g2 && key_less(a1, b1, a2, b2));
}

// warp argmax of (gbits desc, key asc) + sum of `acc`; result valid in lane 0
struct Best {
    unsigned long long g, a, b;
    long long slot;
};
__device__ __forceinline__ void warp_best(Best &x) {
    for (int off = 16; off > 0; off >>= 1) {
        Best y;
        y.g = __shfl_down_sync(0xffffffffu, x.g, off);
        y.a = __shfl_down_sync(0xffffffffu, x.a, off);
        y.b = __shfl_down_sync(0xffffffffu, x.b, off);
        y.slot = __shfl_down_sync(0xffffffffu, x.slot, off);
        if (better(y.g, y.a, y.b, x.g, x.a, x.b)) x = y;
    }
}
__device__ __forceinline__ double warp_sum(double x) {
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    return x;
}
__device__ __forceinline__ int warp_isum(int x) {
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    return x;
}

__device__ __forceinline__ CdPartial load_partial(const CdPartial *p) {
    CdPartial x;
    x.gather = __ldcg(&p->gather);
    x.gbits = __ldcg(&p->gbits);
    x.ka = __ldcg(&p->ka);
    x.kb = __ldcg(&p->kb);
    x.slot = __ldcg(&p->slot);
    x.elements = __ldcg(&p->elements);
    x.applied = __ldcg(&p->applied);
    x.dropped = __ldcg(&p->dropped);
    x.inserted = __ldcg(&p->inserted);
    return x;
}

constexpr int kCdThreads = 256;
constexpr int kCdWarps = kCdThreads / 32;

__global__ void __launch_bounds__(kCdThreads) k_cd_iter(Problem P, IterState *st, CdPartial *part) {
    __shared__ ColLists L;
    __shared__ unsigned long long s_a, s_b;
    __shared__ long long s_slot;
    __shared__ int s_skip, s_last, s_forced;
    __shared__ double s_eta, s_ci_old, s_ci_new, s_Hii;
    __shared__ dd s_mu, s_alpha;
    __shared__ Best r_best[kCdWarps];
    __shared__ double r_gather[kCdWarps];
    __shared__ int r_cnt[4][kCdWarps];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        volatile IterState *vs = st;
        s_skip = vs->done | vs->status;
        s_a = st->sel_a;
        s_b = st->sel_b;
        s_slot = st->sel_slot;
        s_forced = st->forced_eta_one;
    }
    __syncthreads();
    if (s_skip) return;
    const unsigned long long A = s_a, B = s_b;
    build_lists(L, P.N, A, B);
    __syncthreads();

    // ---- prologue: H_ii, step size, scalars (identical in every CTA) ----
    if (warp == 0) {
        double Hii = diag_warp(P, L);
        if (lane == 0) {
            Slot *si = P.table + s_slot;
            double c = __ldcg(&si->c), b = __ldcg(&si->bv);
            dd mu = st->mu, alpha = st->alpha;
            double eta;
            if (s_forced) {
                eta = 1.0;
            } else {
                double v1 = 4.0 * b + 4.0 * mu.hi * c;
                double v2 = 2.0 * Hii + 4.0 * c * c + 2.0 * mu.hi;
                double v3 = 4.0 * c;
                eta = line_search(v1, v2, v3);
            }
            // mu += 2 eta c + eta^2 ; alpha += 2 eta b + eta^2 H_ii
            dd e2 = dd_two_prod(eta, eta);
            dd mu_n = dd_add(dd_add(mu, dd_two_prod(2.0 * eta, c)), e2);
            dd al_n = dd_add(dd_add(alpha, dd_two_prod(2.0 * eta, b)), dd_mul_d(e2, Hii));
            s_eta = eta;
            s_ci_old = c;
            s_ci_new = c + eta;
            s_Hii = Hii;
            s_mu = mu_n;
            s_alpha = al_n;
        }
    }
    __syncthreads();
    const double eta = s_eta, mu = s_mu.hi, tau = P.tau;
    const long long nh = P.doubles_vanish ? P.seg[2] : P.seg[5];

    // ---- scatter / gather / argmax over this CTA's elements ----
    Best best{0ull, ~0ull, ~0ull, -1};
    double gather = 0.0;
    int n_el = 0, n_app = 0, n_drop = 0, n_ins = 0;
    for (long long e = 1 + (long long)blockIdx.x * kCdThreads + tid; e < nh; e += (long long)gridDim.x * kCdThreads) {
        unsigned long long oa, ob;
        double H = column_element(P, L, A, B, e, oa, ob);
        if (H == 0.0) continue;
        ++n_el;
        double v = eta * H;
        bool big = fabs(v) >= tau;
        bool ins = false;
        long long s = table_find(P, st, oa, ob, big, &ins);
        if (s == -2) break;
        if (s < 0) { ++n_drop; continue; }
        Slot *sj = P.table + s;
        double cj = __ldcg(&sj->c);
        if (cj != 0.0 || big) {
            double old = atomicAdd(&sj->bv, v);
            double bn = old + v;
            ++n_app;
            n_ins += ins ? 1 : 0;
            unsigned long long gb = (unsigned long long)__double_as_longlong(fabs(4.0 * (bn + mu * cj)));
            if (better(gb, oa, ob, best.g, best.a, best.b)) best = Best{gb, oa, ob, s};
            gather = fma(H, cj, gather);
        } else {
            ++n_drop;
        }
    }
    warp_best(best);
    gather = warp_sum(gather);
    n_el = warp_isum(n_el);
    n_app = warp_isum(n_app);
    n_drop = warp_isum(n_drop);
    n_ins = warp_isum(n_ins);
    if (lane == 0) {
        r_best[warp] = best;
        r_gather[warp] = gather;
        r_cnt[0][warp] = n_el;
        r_cnt[1][warp] = n_app;
        r_cnt[2][warp] = n_drop;
        r_cnt[3][warp] = n_ins;
    }
    __syncthreads();
    if (tid == 0) {
        Best b = r_best[0];
        double gs = r_gather[0];
        int c0 = r_cnt[0][0], c1 = r_cnt[1][0], c2 = r_cnt[2][0], c3 = r_cnt[3][0];
        for (int w = 1; w < kCdWarps; ++w) {
            if (better(r_best[w].g, r_best[w].a, r_best[w].b, b.g, b.a, b.b)) b = r_best[w];
            gs += r_gather[w];
            c0 += r_cnt[0][w]; c1 += r_cnt[1][w]; c2 += r_cnt[2][w]; c3 += r_cnt[3][w];
        }
        CdPartial pp;
        pp.gather = gs; pp.gbits = b.g; pp.ka = b.a; pp.kb = b.b; pp.slot = b.slot;
        pp.elements = c0; pp.applied = c1; pp.dropped = c2; pp.inserted = c3;
        part[blockIdx.x] = pp;
        __threadfence();
        unsigned int t = atomicAdd(&st->arrive, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ---- tail: the last CTA to arrive finishes the iteration ----
    Best tb{0ull, ~0ull, ~0ull, -1};
    double tg = 0.0;
    long long tc[4] = {0, 0, 0, 0};
    for (int q = tid; q < (int)gridDim.x; q += kCdThreads) {   // fixed order per thread
        CdPartial pp = load_partial(part + q);
        if (better(pp.gbits, pp.ka, pp.kb, tb.g, tb.a, tb.b)) tb = Best{pp.gbits, pp.ka, pp.kb, pp.slot};
        tg += pp.gather;
        tc[0] += pp.elements; tc[1] += pp.applied; tc[2] += pp.dropped; tc[3] += pp.inserted;
    }
    warp_best(tb);
    tg = warp_sum(tg);
    for (int k = 0; k < 4; ++k)
        for (int off = 16; off > 0; off >>= 1) tc[k] += __shfl_down_sync(0xffffffffu, tc[k], off);
    __shared__ long long r_tc[4][kCdWarps];
    if (lane == 0) {
        r_best[warp] = tb;
        r_gather[warp] = tg;
        for (int k = 0; k < 4; ++k) r_tc[k][warp] = tc[k];
    }
    __syncthreads();
    if (tid != 0) return;
    Best b = r_best[0];
    double gsum = r_gather[0];
    long long cnt[4] = {r_tc[0][0], r_tc[1][0], r_tc[2][0], r_tc[3][0]};
    for (int w = 1; w < kCdWarps; ++w) {
        if (better(r_best[w].g, r_best[w].a, r_best[w].b, b.g, b.a, b.b)) b = r_best[w];
        gsum += r_gather[w];
        for (int k = 0; k < 4; ++k) cnt[k] += r_tc[k][w];
    }
    // recalculated b_i = H_ii c_i + sum_{j != i} H_ji c_j with the updated c
    const double ci = s_ci_new;
    const double bi = fma(s_Hii, ci, gsum);
    Slot *si = P.table + s_slot;
    si->c = ci;
    si->bv = bi;
    unsigned long long gi_bits = (unsigned long long)__double_as_longlong(fabs(4.0 * (bi + mu * ci)));
    if (better(gi_bits, A, B, b.g, b.a, b.b)) b = Best{gi_bits, A, B, s_slot};
    if (!isfinite(__longlong_as_double((long long)b.g)) || !isfinite(eta) || !isfinite(s_mu.hi) ||
        !isfinite(s_alpha.hi))
        set_status(st, kErrNonfinite);
    if (b.slot < 0 || b.slot >= P.capacity) {   // cannot happen: i itself is always a candidate
        set_status(st, kErrArg);
        b = Best{gi_bits, A, B, s_slot};
    }
    st->sel_a = b.a;
    st->sel_b = b.b;
    st->sel_slot = b.slot;
    st->mu = s_mu;
    st->alpha = s_alpha;
    st->energy = dd_div_to_d(s_alpha, s_mu);
    st->last_eta = eta;
    st->last_a = A;
    st->last_b = B;
    if (s_forced) {
        st->forced_eta_one = 0;
    } else {
        st->iterations += 1;
        st->dx = P.theta * st->dx + (1.0 - P.theta) * fabs(eta);
        if (P.dx_threshold > 0.0 && st->dx < P.dx_threshold) st->done = 1;
    }
    if (s_ci_old == 0.0 && ci != 0.0) st->nnz_c += 1;
    if (s_ci_old != 0.0 && ci == 0.0) st->nnz_c -= 1;
    const int diag_nz = (s_Hii != 0.0) ? 1 : 0;
    st->elements += cnt[0] + diag_nz;
    st->applied += cnt[1] + diag_nz;
    st->dropped += cnt[2];
    st->inserted += cnt[3];
    st->n_slots += cnt[3];
    st->last_column = cnt[0] + diag_nz;
    if (st->n_slots > P.max_entries) set_status(st, kErrTableFull);
    st->arrive = 0u;
}

// ---------------------------------------------------------------------------
// get_column: every nonzero element of the column of {A, B}, compacted with
// an atomic counter (order unspecified).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_column(Problem P, unsigned long long A, unsigned long long B,
                                                 unsigned long long *keys, double *vals, long long cap,
                                                 unsigned long long *counter) {
    __shared__ ColLists L;
    build_lists(L, P.N, A, B);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        double d = diag_warp(P, L);
        if (threadIdx.x == 0 && d != 0.0) {
            unsigned long long pos = atomicAdd(counter, 1ull);
            if ((long long)pos < cap) { keys[2 * pos] = A; keys[2 * pos + 1] = B; vals[pos] = d; }
        }
    }
    const long long nh = P.seg[5];
    for (long long e = 1 + (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nh;
         e += (long long)gridDim.x * blockDim.x) {
        unsigned long long oa, ob;
        double H = column_element(P, L, A, B, e, oa, ob);
        if (H == 0.0) continue;
        unsigned long long pos = atomicAdd(counter, 1ull);
        if ((long long)pos < cap) { keys[2 * pos] = oa; keys[2 * pos + 1] = ob; vals[pos] = H; }
    }
}

// ---------------------------------------------------------------------------
// Export of the stored entries (true values = stored * scale).
// ---------------------------------------------------------------------------
__global__ void k_export(Problem P, const IterState *st, unsigned long long *keys, double *c, double *b,
                         long long cap, unsigned long long *counter) {
    const double s = st->scale.hi + st->scale.lo;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.capacity;
         i += (long long)gridDim.x * blockDim.x) {
        Slot sl = P.table[i];
        if (sl.a == 0ull && sl.b == 0ull) continue;
        unsigned long long pos = atomicAdd(counter, 1ull);
        if ((long long)pos < cap) {
            keys[2 * pos] = sl.a;
            keys[2 * pos + 1] = sl.b;
            if (c) c[pos] = sl.c * s;
            if (b) b[pos] = sl.bv * s;
        }
    }
}

// ---------------------------------------------------------------------------
// Exact Rayleigh quotient: for every stored i with c_i != 0, (Hc)_i from a
// fresh column (lookups only); per-CTA partial sums, reduced in fixed order.
// ---------------------------------------------------------------------------
__global__ void k_list_nonzero(Problem P, long long *list, long long cap, unsigned long long *counter) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.capacity;
         i += (long long)gridDim.x * blockDim.x) {
        Slot sl = P.table[i];
        if ((sl.a | sl.b) == 0ull || sl.c == 0.0) continue;
        unsigned long long pos = atomicAdd(counter, 1ull);
        if ((long long)pos < cap) list[pos] = i;
    }
}

__global__ void __launch_bounds__(256) k_rq_partial(Problem P, IterState *st, const long long *list, long long cap,
                                                    const unsigned long long *count, double *partial) {
    __shared__ ColLists L;
    __shared__ double r[2][8];
    __shared__ unsigned long long s_a, s_b;
    __shared__ double s_ci, s_diag;
    const long long n = (long long)*count < cap ? (long long)*count : cap;
    const long long nh = P.doubles_vanish ? P.seg[2] : P.seg[5];
    double num_acc = 0.0, den_acc = 0.0;   // meaningful in thread 0
    for (long long k = blockIdx.x; k < n; k += gridDim.x) {
        if (threadIdx.x == 0) {
            Slot sl = P.table[list[k]];
            s_a = sl.a; s_b = sl.b; s_ci = sl.c;
        }
        __syncthreads();
        build_lists(L, P.N, s_a, s_b);
        __syncthreads();
        if (threadIdx.x < 32) {
            double d = diag_warp(P, L);
            if (threadIdx.x == 0) s_diag = d;
        }
        double acc = 0.0;
        for (long long e = 1 + threadIdx.x; e < nh; e += blockDim.x) {
            unsigned long long oa, ob;
            double H = column_element(P, L, s_a, s_b, e, oa, ob);
            if (H == 0.0) continue;
            bool ins = false;
            long long s = table_find(P, st, oa, ob, false, &ins);
            if (s < 0) continue;
            acc = fma(H, P.table[s].c, acc);
        }
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) r[0][threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += r[0][w];
            double hc = fma(s_diag, s_ci, t);
            num_acc = fma(s_ci, hc, num_acc);
            den_acc = fma(s_ci, s_ci, den_acc);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = num_acc;
        partial[2 * blockIdx.x + 1] = den_acc;
    }
}

__global__ void k_rq_final(const double *partial, int n, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < n; ++i) { a += partial[2 * i]; b += partial[2 * i + 1]; }
    out[0] = a / b;
}

// ---------------------------------------------------------------------------
// Set-up kernels
// ---------------------------------------------------------------------------
// Validate finiteness and 8-fold symmetry of g (relative tolerance), then make
// every image hold the value of the canonical element, so that identities such
// as (ia|ii) - (ii|ia) = 0 hold exactly.
__global__ void k_validate_g(double *g, int N, double tol, int *status) {
    const long long n4 = (long long)N * N * N * N;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += (long long)gridDim.x * blockDim.x) {
        int s = (int)(t % N), r = (int)((t / N) % N), q = (int)((t / N / N) % N), p = (int)(t / N / N / N);
        int p1 = p > q ? p : q, q1 = p > q ? q : p;
        int r1 = r > s ? r : s, s1 = r > s ? s : r;
        int pq = p1 * (p1 + 1) / 2 + q1, rs = r1 * (r1 + 1) / 2 + s1;
        long long canon = pq >= rs ? ((((long long)p1 * N + q1) * N + r1) * N + s1)
                                   : ((((long long)r1 * N + s1) * N + p1) * N + q1);
        double x = g[t], y = g[canon];
        if (!isfinite(x)) { atomicCAS(status, 0, kErrNonfinite); continue; }
        if (fabs(x - y) > tol * fmax(1.0, fabs(y))) atomicCAS(status, 0, kErrArg);
    }
}
__global__ void k_canonicalize_g(double *g, int N) {
    const long long n4 = (long long)N * N * N * N;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += (long long)gridDim.x * blockDim.x) {
        int s = (int)(t % N), r = (int)((t / N) % N), q = (int)((t / N / N) % N), p = (int)(t / N / N / N);
        int p1 = p > q ? p : q, q1 = p > q ? q : p;
        int r1 = r > s ? r : s, s1 = r > s ? s : r;
        int pq = p1 * (p1 + 1) / 2 + q1, rs = r1 * (r1 + 1) / 2 + s1;
        long long canon = pq >= rs ? ((((long long)p1 * N + q1) * N + r1) * N + s1)
                                   : ((((long long)r1 * N + s1) * N + p1) * N + q1);
        if (canon != t) g[t] = g[canon];
    }
}
// a canonical element is never overwritten, so the order of the writes does not matter

__global__ void k_validate_h(const double *h, int N, double tol, int *status) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * N; t += gridDim.x * blockDim.x) {
        int p = t / N, q = t % N;
        double x = h[t], y = h[q * N + p];
        if (!isfinite(x)) { atomicCAS(status, 0, kErrNonfinite); continue; }
        if (fabs(x - y) > tol * fmax(1.0, fabs(y))) atomicCAS(status, 0, kErrArg);
    }
}
__global__ void k_symmetrize_h(double *h, int N) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * N; t += gridDim.x * blockDim.x) {
        int p = t / N, q = t % N;
        if (p < q) h[t] = h[q * N + p];
    }
}

// J_pq = (pp|qq), K_pq = (pq|qp); flag = 1 if some (pq|rs) with p != q and r != s is nonzero
__global__ void k_jk(const double *g, int N, double *J, double *K, int *has_doubles) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * N; t += gridDim.x * blockDim.x) {
        int p = t / N, q = t % N;
        J[t] = g[(((size_t)p * N + p) * N + q) * N + q];
        K[t] = g[(((size_t)p * N + q) * N + q) * N + p];
    }
    const long long n4 = (long long)N * N * N * N;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += (long long)gridDim.x * blockDim.x) {
        int s = (int)(t % N), r = (int)((t / N) % N), q = (int)((t / N / N) % N), p = (int)(t / N / N / N);
        if (p != q && r != s && g[t] != 0.0) atomicExch(has_doubles, 1);
    }
}

// Insert the start determinant and set the state for the initialisation launch
// (c = e_ref reached from c = 0 with eta = 1: mu = 1, alpha = H_ref,ref).
__global__ void k_init_state(Problem P, IterState *st, unsigned long long A, unsigned long long B) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bool ins = false;
    long long s = table_find(P, st, A, B, true, &ins);
    st->sel_a = A;
    st->sel_b = B;
    st->sel_slot = s < 0 ? 0 : s;
    if (s < 0) set_status(st, kErrTableFull);
    st->forced_eta_one = 1;
    st->done = 0;
    st->arrive = 0u;
    st->mu = dd_from(0.0);
    st->alpha = dd_from(0.0);
    st->scale = dd_from(1.0);
    st->dx = 0.0;
    st->energy = 0.0;
    st->iterations = 0;
    st->last_eta = 0.0;
    st->last_a = A;
    st->last_b = B;
    st->nnz_c = 0;
    st->n_slots = 1;
    st->last_column = 0;
    st->elements = 0;
    st->applied = 0;
    st->dropped = 0;
    st->inserted = 1;
}

// ---------------------------------------------------------------------------
// Launch wrappers (host)
// ---------------------------------------------------------------------------
cudaError_t launch_cd_iter(const Problem &P, IterState *st, CdPartial *part, int grid, cudaStream_t s) {
    k_cd_iter<<<grid, kCdThreads, 0, s>>>(P, st, part);
    return cudaGetLastError();
}
int cd_threads() { return kCdThreads; }

cudaError_t launch_column(const Problem &P, unsigned long long A, unsigned long long B, unsigned long long *keys,
                          double *vals, long long cap, unsigned long long *counter, cudaStream_t s) {
    long long nh = P.seg[5];
    int grid = (int)((nh + 255) / 256);
    if (grid < 1) grid = 1;
    if (grid > 4096) grid = 4096;
    k_column<<<grid, 256, 0, s>>>(P, A, B, keys, vals, cap, counter);
    return cudaGetLastError();
}

cudaError_t launch_export(const Problem &P, const IterState *st, unsigned long long *keys, double *c, double *b,
                          long long cap, unsigned long long *counter, cudaStream_t s) {
    long long grid = (P.capacity + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    k_export<<<(int)grid, 256, 0, s>>>(P, st, keys, c, b, cap, counter);
    return cudaGetLastError();
}

cudaError_t launch_rq(const Problem &P, IterState *st, long long *list, long long cap, unsigned long long *counter,
                      double *partial, int nblocks, double *out, cudaStream_t s) {
    long long grid = (P.capacity + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    k_list_nonzero<<<(int)grid, 256, 0, s>>>(P, list, cap, counter);
    k_rq_partial<<<nblocks, 256, 0, s>>>(P, st, list, cap, counter, partial);
    k_rq_final<<<1, 32, 0, s>>>(partial, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_setup(double *h, double *g, int N, double *J, double *K, int *status, int *has_doubles,
                         cudaStream_t s) {
    long long n4 = (long long)N * N * N * N;
    int grid = (int)((n4 + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_validate_h<<<4, 256, 0, s>>>(h, N, 1e-12, status);
    k_validate_g<<<grid, 256, 0, s>>>(g, N, 1e-12, status);
    k_symmetrize_h<<<4, 256, 0, s>>>(h, N);
    k_canonicalize_g<<<grid, 256, 0, s>>>(g, N);
    k_jk<<<grid, 256, 0, s>>>(g, N, J, K, has_doubles);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const Problem &P, IterState *st, unsigned long long A, unsigned long long B,
                              cudaStream_t s) {
    k_init_state<<<1, 32, 0, s>>>(P, st, A, B);
    return cudaGetLastError();
}

}  // namespace cdfci
