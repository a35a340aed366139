// CUDA kernels of libcdfci (sm_103a).
//
// The m = 1 iteration (Algorithm 1) runs inside a persistent loop kernel that
// performs many iterations per launch on G CTAs (one per SM): k_cd_loop, a
// thread-block cluster (G <= 16, partials exchanged through distributed shared
// memory), or k_cd_loop_grid, a cooperative grid (G > 16, partials through
// global memory and a software grid barrier).  Per iteration:
//   1. warp 0 (the control warp) of every CTA reads the partials of the
//      previous iteration of every CTA and reduces them in a fixed order: the
//      recalculated b of the previous coordinate (Eq. recalculate-b) and the
//      argmax of |b_j + mu c_j| over the previous column and that coordinate
//      (Eq. choose-i; the factor 4 does not change the argmax) -> i, identical
//      in every CTA;
//   2. every warp builds the orbital lists of i; the element warps load the
//      terms of the CTA's single excitations, build the single-excitation
//      tables, decode their share of the column (Slater-Condon, Eq. entry),
//      issue the 32-byte slot loads and evaluate the elements (the singles'
//      O(n) sums spread over the CTA through a shared-memory term table);
//   3. meanwhile the control warp computes H_ii (from shared-memory copies of
//      diag(h), J and K) and one lane the step size eta (appendix);
//   4. every element thread applies b_j += eta H_ji with the compression rule
//      (c_j != 0 or |eta H_ji| >= tau), inserting absent keys with a 16-byte
//      CAS, and accumulates the gather sum_j H_ji c_j and its best candidate;
//   5. the control warp combines the CTA's partial and writes it while two
//      lanes of warp 1 update mu and alpha (double-double); cluster or grid
//      barrier.
// In an m = 1 column every j occurs once, so each b_j has a single writer:
// plain loads and stores, no atomics.  The previous coordinate's slot is
// written by the thread whose excitation equals it, with the recalculated b.
#include <cooperative_groups.h>

#include <algorithm>

#include "cdfci_internal.cuh"
#include "cdfci_kernels.h"

namespace cdfci {

__device__ __forceinline__ bool better(unsigned long long g1, unsigned long long a1, unsigned long long b1,
                                       unsigned long long g2, unsigned long long a2, unsigned long long b2) {
    return g1 > g2 || (g1 == g2 && key_less(a1, b1, a2, b2));
}

// a candidate of the argmax of (gbits desc, key asc)
struct Best {
    unsigned long long g, a, b;
    long long slot;
};
__device__ __forceinline__ double warp_sum(double x) {
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    return x;
}

constexpr int kCdThreads = 384;                 // threads per CTA of the cluster
constexpr int kCdWarps = kCdThreads / 32;
constexpr int kCdMaxE = 3;                      // elements whose slot loads a thread keeps in flight
constexpr int kCdMaxCluster = 16;

// One pending column element of a thread.
struct Elem {
    unsigned long long ka, kb;         // key D'
    ElemIdx ix;
    double H;
    ulonglong2 k0;                     // first probed slot: key ...
    double2 cb0;                       // ... and (c, b)
    long long pos;                     // probe position
    int state;                         // 0 none, 1 found, 2 absent (pos = first empty slot), 3 previous coordinate,
                                       // 4 first probe issued, not yet resolved
};

// Dynamic shared memory of the m = 1 loop kernels: the column's single-
// excitation tables (alpha then beta), J and K, the diagonal of h, the pairs
// of occupied positions, and the term table of the singles a CTA evaluates
// term-parallel: 32-element blocks of the single segment, at most as many as a
// thread's first round of elements covers and as fit in kTermBytes, each
// holding 32 x (n_alpha + n_beta + 1) entries.
constexpr int kTermBytes = 32 * 1024;
constexpr int kCdMaxDynSmem = 200 * 1024;   // N <= 64: <= 49 KB tables, 64 KB J and K, 16 KB pairs, 32 KB terms
struct CdSmem {
    size_t off_j, off_k, off_hd, off_pairs, off_t, bytes;
    int npairs;                        // unordered pairs u < w of the n_alpha + n_beta occupied positions
    int tb_max;                        // blocks in the term table (the most any CTA owns, G = 1)
};
__host__ __device__ inline CdSmem cd_smem_layout(const Problem &P) {
    CdSmem L;
    const size_t tab = (size_t)(P.na * P.va + P.nb * P.vb + 1) * sizeof(SingleEnt);
    const int nocc = P.na + P.nb;
    L.npairs = nocc * (nocc - 1) / 2;
    L.off_j = (tab + 15) & ~(size_t)15;
    L.off_k = L.off_j + (size_t)P.N * P.N * sizeof(double);
    L.off_hd = L.off_k + (size_t)P.N * P.N * sizeof(double);
    L.off_pairs = L.off_hd + (size_t)P.N * sizeof(double);
    L.off_t = (L.off_pairs + (size_t)L.npairs * sizeof(unsigned short) + 15) & ~(size_t)15;
    const int nqs = (int)((P.seg[2] - P.seg[0] + 31) / 32);
    const int cap = kTermBytes / (32 * (int)sizeof(double) * (nocc + 1));
    int tb = nqs < (kCdWarps - 1) * kCdMaxE ? nqs : (kCdWarps - 1) * kCdMaxE;
    if (tb > (cap > 1 ? cap : 1)) tb = cap > 1 ? cap : 1;
    L.tb_max = tb;
    L.bytes = L.off_t + (size_t)tb * 32 * (nocc + 1) * sizeof(double);
    return L;
}

// Pair table of the occupied positions (alpha 0 .. n_alpha - 1, then beta):
// u | w << 7 | same spin << 14 for u < w, in the order (0,1), (0,2), ...,
// (1,2), ...; filled by the threads of a CTA, u per thread.
__device__ __forceinline__ void fill_pairs(const Problem &P, unsigned short *pairs) {
    const int n = P.na + P.nb;
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
        const int base = u * n - u * (u + 1) / 2;
        for (int w = u + 1; w < n; ++w)
            pairs[base + (w - u - 1)] = (unsigned short)(u | (w << 7) | (((u < P.na) == (w < P.na)) ? 1 << 14 : 0));
    }
}

// Diagonal element (Eq. entry, i = j) by one warp from shared-memory copies of
// diag(h), J and K: sum_p h_pp + sum over unordered occupied pairs of J - K
// (same spin) or J (opposite spins).  Lane l takes pairs l + 32 r into four
// partial sums (r mod 4) and the h terms of positions l, l + 32, ...; the lane
// values are combined by a shuffle-down tree, every lane returns the result.
__device__ __forceinline__ double diag_pairs_warp(const Problem &P, const ColLists &L, const double *sHd,
                                                  const double *sJ, const double *sK, const unsigned short *pairs,
                                                  int npairs) {
    const int lane = threadIdx.x & 31, N = P.N, na = P.na, n = P.na + P.nb;
    double y0 = 0.0, y1 = 0.0, y2 = 0.0, y3 = 0.0;
    for (int k0 = lane; k0 < npairs; k0 += 128) {
        double t[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = k0 + 32 * r;
            t[r] = 0.0;
            if (k < npairs) {
                const unsigned pr = pairs[k];
                const int u = pr & 0x7f, w = (pr >> 7) & 0x7f;
                const int p = u < na ? L.occA[u] : L.occB[u - na];
                const int q = w < na ? L.occA[w] : L.occB[w - na];
                const double jv = sJ[p * N + q];
                t[r] = (pr >> 14) ? jv - sK[p * N + q] : jv;
            }
        }
        y0 += t[0]; y1 += t[1]; y2 += t[2]; y3 += t[3];
    }
    double x = 0.0;
    for (int u = lane; u < n; u += 32) x += sHd[u < na ? L.occA[u] : L.occB[u - na]];
    x += (y0 + y1) + (y2 + y3);
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    return __shfl_sync(0xffffffffu, x, 0);
}

// Address of entry idx = ls * (nocc + 1) + kk of the CTA's term table: single
// ls (block ls / 32 of this CTA's share, lane ls % 32); kk < nocc: the term of
// occupied spin-orbital kk in spin-orbital order (the n_alpha alpha orbitals,
// then the n_beta beta ones; W3 for the single's own spin, V3 for the other);
// kk = nocc: h_ia.  The single's orbitals come from the lists, so the loads do
// not wait for the singles tables.  Past the last single a valid dummy address
// (h_00).
__device__ __forceinline__ const double *single_term_ptr(const Problem &P, const ColLists &L, int rank, int G,
                                                         int nocc, long long nsing, int idx) {
    const int ls = idx / (nocc + 1), kk = idx - ls * (nocc + 1);
    const long long s = 32ll * (rank + (long long)G * (ls >> 5)) + (ls & 31);
    if (s >= nsing) return P.h;
    const int nsa = P.na * P.va;
    const bool alpha = s < nsa;
    const unsigned sl = (unsigned)(alpha ? s : s - nsa);
    const int o = (int)fdiv(sl, alpha ? P.mg_va : P.mg_vb);
    const int w = (int)sl - o * (alpha ? P.va : P.vb);
    const int i = alpha ? L.occA[o] : L.occB[o];
    const int a = alpha ? L.virA[w] : L.virB[w];
    if (kk == nocc) return P.h + i * P.N + a;
    const bool k_alpha = kk < P.na;
    const int k = k_alpha ? L.occA[kk] : L.occB[kk - P.na];
    return (k_alpha == alpha ? P.W3 : P.V3) + ((size_t)(i * P.N + a) * P.N + k);
}

// A single's value from its row of terms: h_ia, then the nocc terms in the
// row's order, one running sum (the order of element_value).
__device__ __forceinline__ double single_sum(const double *row, int nocc, unsigned long long sgn) {
    double v = row[nocc];
    for (int k = 0; k < nocc; ++k) v += row[k];
    return apply_parity(v, sgn);
}

// Decode element e (singles and opposite-spin doubles from the tables) and
// issue the load of its first probe slot (32 bytes).
// A whole 32-byte slot {key, c, b} in one request (two 16-byte loads of one
// slot are two DRAM accesses on this memory system); L2 only.
__device__ __forceinline__ void ld_slot32(const Slot *s, ulonglong2 &k, double2 &cb) {
    unsigned long long c, b;
    asm volatile("ld.global.cg.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(k.x), "=l"(k.y), "=l"(c), "=l"(b) : "l"(s));
    cb.x = __longlong_as_double((long long)c);
    cb.y = __longlong_as_double((long long)b);
}

__device__ __forceinline__ void issue_elem(const Problem &P, const ColLists &L, const SingleEnt *tabA,
                                           const SingleEnt *tabB, unsigned long long iA, unsigned long long iB,
                                           unsigned long long hA, unsigned long long hB, long long e, long long nh,
                                           bool have_prev, unsigned long long pA, unsigned long long pB, Elem &x) {
    x.state = 0;
    if (e >= nh) return;
    unsigned long long h;
    if (e >= P.seg[4]) {                                   // opposite-spin double from two singles
        const unsigned idx = (unsigned)(e - P.seg[4]);
        const unsigned sa = fdiv(idx, P.mg_nsb);
        const unsigned sb = idx - sa * (unsigned)(P.nb * P.vb);
        const SingleEnt ea = tabA[sa], eb = tabB[sb];
        if (!k_conserved(P, (ea.info >> 24) & 0xff, (eb.info >> 24) & 0xff)) return;   // zero: momentum
        x.ka = ea.key;
        x.kb = eb.key;
        h = ea.h ^ eb.h;
        x.ix.kind = 4;
        x.ix.sgn = (unsigned long long)((ea.info ^ eb.info) & 1);
        x.ix.gidx = ea.goff + eb.goff;
    } else if (e < P.seg[2]) {                             // single
        const bool alpha = e < P.seg[1];
        const SingleEnt es = alpha ? tabA[e - P.seg[0]] : tabB[e - P.seg[1]];
        x.ka = alpha ? es.key : iA;
        x.kb = alpha ? iB : es.key;
        h = alpha ? (es.h ^ hB) : (hA ^ es.h);
        x.ix.kind = alpha ? 0 : 1;
        x.ix.sgn = (unsigned long long)(es.info & 1);
        x.ix.i = (es.info >> 8) & 0xff;
        x.ix.a = (es.info >> 16) & 0xff;
        x.ix.gidx = -1;
    } else {                                               // same-spin double
        decode_element(P, L, iA, iB, e, x.ka, x.kb, x.ix);
        h = (x.ix.kind == 2) ? (hash_alpha(x.ka) ^ hB) : (hA ^ hash_beta(x.kb));
    }
    if (have_prev && x.ka == pA && x.kb == pB) { x.state = 3; return; }
    x.pos = (long long)(h & P.mask);
    const Slot *s = P.table + x.pos;
    ld_slot32(s, x.k0, x.cb0);
    x.state = 4;
}

// Finish the lookup of an issued element: compare the first slot, probe on if
// needed.  Sets state 1 (found: c, bv), 2 (absent at pos) or 0 (value zero or
// error, *err set).
__device__ __forceinline__ void resolve_elem(const Problem &P, IterState *st, Elem &x, int *err) {
    if (x.state != 4) return;
    if (is_zero(x.H)) { x.state = 0; return; }
    const bool both_nonzero = (P.na > 0) && (P.nb > 0);
    unsigned long long p = (unsigned long long)x.pos;
    ulonglong2 k = x.k0;
    double2 cb = x.cb0;
    for (int probe = 0; probe < P.max_probe; ++probe) {
        int spins = 0;
        while (both_nonzero && ((k.x == 0ull) != (k.y == 0ull))) {
            if (++spins > (1 << 20)) { set_status(st, kErrTimeout); *err = 1; x.state = 0; return; }
            ld_slot32(P.table + p, k, cb);
        }
        if (k.x == x.ka && (k.y & kKeyMaskB) == x.kb) { x.pos = (long long)p; x.cb0 = cb; x.state = 1; return; }
        if (k.x == 0ull && k.y == 0ull) { x.pos = (long long)p; x.state = 2; return; }
        p = (p + 1) & P.mask;
        ld_slot32(P.table + p, k, cb);
    }
    set_status(st, kErrTableFull);
    *err = 1;
    x.state = 0;
}

// Claim an empty slot for a key that no other thread inserts concurrently (in
// an m = 1 column every determinant occurs once), starting at `pos`.
__device__ __forceinline__ long long claim_slot(const Problem &P, IterState *st, unsigned long long a,
                                                unsigned long long b, long long pos, int *err) {
    unsigned long long p = (unsigned long long)pos;
    for (int probe = 0; probe < P.max_probe; ++probe) {
        unsigned long long oa, ob;
        cas128(&P.table[p].a, 0ull, 0ull, a, b, oa, ob);
        if (oa == 0ull && ob == 0ull) return (long long)p;
        p = (p + 1) & P.mask;
    }
    set_status(st, kErrTableFull);
    *err = 1;
    return -1;
}

// The coordinate chosen for an iteration and what every warp needs about it.
struct Sel {
    unsigned long long iA, iB;
    long long islot;
    double bi, ci;
    unsigned long long pA, pB;         // previous coordinate (its b is pending)
    long long pslot;
    double pb, pc;
    double eta, mu_g;                  // step size; mu used in the gradients of this column
    double feta;                       // forced step: the given eta
    int have_prev, forced, stop, bad;
};

// Cluster-wide state kept in shared memory (identical in every CTA).
struct LoopState {
    unsigned long long pA, pB;
    long long pslot;
    double pc, pHii, pmu_g, peta;      // previous coordinate: c after its update, H_ii, the mu of its column, eta
    dd mu, alpha;
    double dx;
    long long iterations, nnz_c, n_slots, elements, applied, dropped, inserted, last_column;
    unsigned long long fa, fb;         // forced next coordinate and its step
    double feta;
    int forced, have_prev, done;
};

// Warp-level combine: argmax of (gbits desc, key asc) with payload (slot, b, c),
// sums of the counters and a lane-ordered sum of the nonzero gather values;
// every lane returns the result.  The maximum of gbits comes from a
// butterfly on gbits alone; only exact ties look at the keys.  The gather's
// fixed shuffle-down tree (skipped when every lane holds 0) runs level by level
// beside the butterfly, so their latencies overlap.
__device__ __forceinline__ void warp_combine(Best &best, double &bb, double &cb, double &gather, int cnt[4], int &err) {
    const bool any_g = __any_sync(0xffffffffu, !is_zero(gather));
    for (int k = 0; k < 4; ++k) cnt[k] = __reduce_add_sync(0xffffffffu, (unsigned)cnt[k]);
    err = (int)__reduce_or_sync(0xffffffffu, (unsigned)err);
    unsigned long long gmax = best.g;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, gmax, off);
        const double t = __shfl_down_sync(0xffffffffu, gather, off);
        if (any_g) gather += t;
        gmax = y > gmax ? y : gmax;
    }
    const unsigned int cand = __ballot_sync(0xffffffffu, best.g == gmax && best.slot >= 0);
    int win = cand ? __ffs(cand) - 1 : 0;
    if (__popc(cand) > 1) {
        unsigned long long wa = __shfl_sync(0xffffffffu, best.a, win), wb = __shfl_sync(0xffffffffu, best.b, win);
        unsigned int rest = cand & (cand - 1);
        while (rest) {
            const int l = __ffs(rest) - 1;
            rest &= rest - 1;
            const unsigned long long la = __shfl_sync(0xffffffffu, best.a, l), lb = __shfl_sync(0xffffffffu, best.b, l);
            if (key_less(la, lb, wa, wb)) { win = l; wa = la; wb = lb; }
        }
    }
    if (cand) {
        best.g = gmax;
        best.a = __shfl_sync(0xffffffffu, best.a, win);
        best.b = __shfl_sync(0xffffffffu, best.b, win);
        best.slot = __shfl_sync(0xffffffffu, best.slot, win);
        bb = __shfl_sync(0xffffffffu, bb, win);
        cb = __shfl_sync(0xffffffffu, cb, win);
    } else {
        best = Best{0ull, ~0ull, ~0ull, -1};
        bb = 0.0;
        cb = 0.0;
    }
    if (any_g) gather = __shfl_sync(0xffffffffu, gather, 0);
}

// Partial exchange of the grid-wide loop (all CTAs co-resident: cooperative
// launch).  At the end of round q every CTA publishes its partial into buffer
// q & 1 as kXchgWords words, each (q mod 2^32) << 32 | one 32-bit half of the
// partial; at the start of round q + 1 the control warps poll those words
// until every one carries q.  The publishing lanes fence after the CTA barrier
// that follows the element warps' table writes (release: those writes, the
// slot of the processed coordinate and the partial become visible together),
// and the readers fence after the poll (acquire), so a one-way pass of the data
// replaces a barrier counter's round trip plus the read of the partials.  A CTA
// publishes round q + 2 into the same buffer only after it has read every
// partial of round q + 1, hence after every CTA has read round q: two buffers
// suffice.  The waits are bounded: on expiry the status becomes
// CDFCI_ERR_TIMEOUT and the loop ends.
constexpr int kXchgSpins = 1 << 21;
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void xchg_publish(unsigned long long *dst, const CdPartial &p, unsigned int q, int lane) {
    if (lane < kXchgWords / 2) {
        const unsigned int *h = reinterpret_cast<const unsigned int *>(&p);
        const unsigned long long w0 = ((unsigned long long)q << 32) | h[2 * lane];
        const unsigned long long w1 = ((unsigned long long)q << 32) | h[2 * lane + 1];
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(dst + 2 * lane), "l"(w0), "l"(w1)
                     : "memory");
    }
}
__device__ __forceinline__ void xchg_load(const unsigned long long *src, unsigned long long (&w)[kXchgWords]) {
#pragma unroll
    for (int k = 0; k < kXchgWords; k += 2)
        asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(w[k]), "=l"(w[k + 1]) : "l"(src + k)
                     : "memory");
}
// true when every word carries round q (the padding word 19 is not checked)
__device__ __forceinline__ bool xchg_check(const unsigned long long (&w)[kXchgWords], unsigned int q) {
    unsigned int bad = 0u;
#pragma unroll
    for (int k = 0; k < kXchgWords - 1; ++k) bad |= (unsigned int)(w[k] >> 32) ^ q;
    return bad == 0u;
}
__device__ __forceinline__ unsigned long long xchg_u64(const unsigned long long (&w)[kXchgWords], int k) {
    return (w[k] & 0xffffffffull) | (w[k + 1] << 32);
}
// the partial from its words (the field order of CdPartial, low half first;
// cdfci_api.cu asserts that layout)
__device__ __forceinline__ CdPartial xchg_unpack(const unsigned long long (&w)[kXchgWords]) {
    CdPartial x;
    x.gather = __longlong_as_double((long long)xchg_u64(w, 0));
    x.gbits = xchg_u64(w, 2);
    x.ka = xchg_u64(w, 4);
    x.kb = xchg_u64(w, 6);
    x.slot = (long long)xchg_u64(w, 8);
    x.bj = __longlong_as_double((long long)xchg_u64(w, 10));
    x.cj = __longlong_as_double((long long)xchg_u64(w, 12));
    x.elements = (int)(unsigned int)w[14];
    x.applied = (int)(unsigned int)w[15];
    x.dropped = (int)(unsigned int)w[16];
    x.inserted = (int)(unsigned int)w[17];
    x.err = (int)(unsigned int)w[18];
    return x;
}
// Warp-wide: polls the partial r (if r < G) of round q in buf into x, then
// fences (acquire); false when the wait expired (uniform over the warp).
__device__ __forceinline__ bool xchg_poll1(const unsigned long long *buf, int G, int r, unsigned int q, CdPartial &x) {
    bool ok = r >= G;
    unsigned long long w[kXchgWords];
    for (int spins = 0;; ++spins) {
        if (!ok) {
            xchg_load(buf + (size_t)r * kXchgWords, w);
            ok = xchg_check(w, q);
        }
        if (__all_sync(0xffffffffu, ok)) break;
        if (spins >= kXchgSpins) return false;
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    if (r < G) x = xchg_unpack(w);
    return true;
}

// A partial written by another SM in this round: read through L2 (an L1 line of
// the same buffer from two rounds ago may be stale).
__device__ __forceinline__ CdPartial ldcg_partial(const CdPartial *p) {
    static_assert(sizeof(CdPartial) % 16 == 0, "CdPartial is read as 16-byte words");
    CdPartial x;
    const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(p);
    ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(&x);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(CdPartial) / 16); ++i) dst[i] = __ldcg(src + i);
    return x;
}

// Fold the partials r = lane, lane + 32, ... (fixed order) into this lane's
// accumulators: the best candidate (larger |g|, then the smaller key), the
// gather sum and the counters.
__device__ __forceinline__ void fold_partial(const CdPartial &x, bool first, Best &bb, double &bj, double &cj,
                                             double &gsum, int cnt[4], int &err) {
    if (first) {
        bb = Best{x.gbits, x.ka, x.kb, x.slot};
        bj = x.bj; cj = x.cj; gsum = x.gather;
        cnt[0] = x.elements; cnt[1] = x.applied; cnt[2] = x.dropped; cnt[3] = x.inserted;
        err = x.err;
        return;
    }
    if (x.slot >= 0 && (bb.slot < 0 || better(x.gbits, x.ka, x.kb, bb.g, bb.a, bb.b))) {
        bb = Best{x.gbits, x.ka, x.kb, x.slot};
        bj = x.bj; cj = x.cj;
    }
    gsum += x.gather;
    cnt[0] += x.elements; cnt[1] += x.applied; cnt[2] += x.dropped; cnt[3] += x.inserted;
    err |= x.err;
}

// Algorithm 1 by one thread-block cluster that keeps running: each iteration
// every CTA scatters a share of the column, writes a partial (best candidate,
// gather, counters) into its own shared memory, and after the cluster barrier
// warp 0 of every CTA reads all partials through distributed shared memory and
// reduces them in a fixed order, so every CTA makes the same choice.  The
// serial steps (H_ii, eta, the double-double scalars) run on single lanes;
// their results reach the other warps through shared memory.  Every exit
// decision uses data all CTAs read identically, so all CTAs reach every
// cluster barrier.
//
// kGrid: the same loop over every CTA of a cooperative launch (more CTAs than
// a cluster holds).  The partials of a round then go through the round-numbered
// exchange buffer xchg (see xchg_publish), which replaces the cluster barrier;
// gpart holds the partials between launches (read in a launch's first round,
// written once every CTA has published its last one).
template <bool kGrid, int kE>
__device__ __forceinline__ void cd_loop_body(const Problem &P, IterState *st, CdRecord *rec, CdPartial *gpart,
                                             unsigned long long *xchg, GridRound *rnd, long long n_iter) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int G = kGrid ? (int)gridDim.x : (int)cluster.num_blocks();
    const int rank = kGrid ? (int)blockIdx.x : (int)cluster.block_rank();
    // grid mode: rounds published by earlier launches (mod 2^32); round q0 + it + 1 is published in
    // iteration it
    const unsigned int q0 = kGrid ? (unsigned int)__ldcg(&rnd->round) : 0u;
    unsigned int n_pub = 0;                      // rounds this launch published (grid mode)
    __shared__ CdPartial spart[2];               // cluster: this CTA's partials (alternating); grid: [0] the last published
    __shared__ ColLists Lw[kCdWarps];
    __shared__ Best r_best[kCdWarps];
    __shared__ double r_bc[kCdWarps][3];
    __shared__ int r_cnt[4][kCdWarps];
    __shared__ Sel sel;
    __shared__ int s_done;
    __shared__ LoopState ls;                     // written by lane 0 of the control warp (warp 0) only
    __shared__ double s_hii;
    __shared__ int s_err;
    __shared__ int s_fins;                       // 1: this CTA inserted the forced coordinate of this step
    __shared__ int s_tmo;                        // grid mode: a wait for the partials expired
    __shared__ CdPartial s_x1[kGrid ? 2 : 1][32];   // grid mode: the partials polled by warps 0 and 1
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const CdSmem lay = cd_smem_layout(P);
    SingleEnt *tabA = reinterpret_cast<SingleEnt *>(s_dyn), *tabB = tabA + P.na * P.va;
    double *sJ = reinterpret_cast<double *>(s_dyn + lay.off_j);
    double *sK = reinterpret_cast<double *>(s_dyn + lay.off_k);
    double *sHd = reinterpret_cast<double *>(s_dyn + lay.off_hd);
    unsigned short *sPairs = reinterpret_cast<unsigned short *>(s_dyn + lay.off_pairs);
    double *sTerm = reinterpret_cast<double *>(s_dyn + lay.off_t);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (rec->done) return;                       // uniform: nothing has synchronised yet
    for (int t = tid; t < P.N * P.N; t += kCdThreads) {
        sJ[t] = __ldg(P.J + t);
        sK[t] = __ldg(P.K + t);
    }
    for (int t = tid; t < P.N; t += kCdThreads) sHd[t] = __ldg(P.h + t * (P.N + 1));
    fill_pairs(P, sPairs);
    if (tid == 0) {
        const CdRecord &R = *rec;
        ls.pA = R.a; ls.pB = R.b; ls.pslot = R.slot;
        ls.pc = R.c_new; ls.pHii = R.Hii; ls.pmu_g = R.mu_g; ls.peta = R.eta;
        ls.mu = R.mu; ls.alpha = R.alpha; ls.dx = R.dx;
        ls.iterations = R.iterations; ls.nnz_c = R.nnz_c; ls.n_slots = R.n_slots; ls.elements = R.elements;
        ls.applied = R.applied; ls.dropped = R.dropped; ls.inserted = R.inserted; ls.last_column = R.last_column;
        ls.fa = R.fa; ls.fb = R.fb; ls.feta = R.feta;
        ls.forced = R.forced; ls.have_prev = R.have_prev; ls.done = 0;
        if (!kGrid) spart[1] = gpart[rank];
        s_err = 0;
        s_done = 0;
        s_fins = 0;
        s_tmo = 0;
    }
    if (kGrid) __syncthreads(); else cluster.sync();

    // Element e - 1 = lane + 32 * (rank + G * (w + W' * j)), w = warp - 1, W' = warps - 1,
    // j = 0, 1, ...: 32 consecutive elements per warp, consecutive warps' worth
    // on different CTAs.  The single excitations (the first elements, each an
    // O(n) sum) thus fill whole warps spread over CTAs: their FP64 sums run
    // with all lanes active.  Warp 0 is the control warp and owns no elements.
    const long long nh = P.doubles_vanish ? P.seg[2] : P.seg[5];
    constexpr int Wp = kCdWarps - 1;
    const long long stride = (long long)G * Wp * 32;
    const long long e0 = warp == 0 ? nh : 1 + lane + 32ll * (rank + (long long)G * (warp - 1));
    // Singles of this CTA (blocks rank, rank + G, ... of the single segment) in
    // the term table: their O(n) sums are spread over all element threads
    // instead of running as one thread's chain of dependent loads.
    const int nocc = P.na + P.nb;
    const long long nsing = P.seg[2] - P.seg[0];
    const int nqs = (int)((nsing + 31) >> 5);
    const int n_own = rank < nqs ? (nqs - 1 - rank) / G + 1 : 0;
    const int tb = min(min(n_own, lay.tb_max), Wp * kE);
    const int nterms = tb * 32 * (nocc + 1);
    int lastp = 1;
    for (long long it = 0; it < n_iter; ++it) {
        const int pin = lastp, pout = lastp ^ 1;
        // ---- choice of i (Eq. choose-i), by the control warp ----
        // every CTA's partial of the last column: lane l of the control warp folds CTAs l, l + 32, ...
        // (all lanes take part in the combine)
        {
        Best bb{0ull, ~0ull, ~0ull, -1};
        double bj = 0.0, cj = 0.0, gsum = 0.0;
        int cnt[4] = {0, 0, 0, 0};
        int err = 0;
        bool tmo = false;
        if (kGrid && it > 0 && warp < 2 && ls.have_prev) {
            // grid mode: warp 0 polls partial r0 + lane, warp 1 partial r0 + 32 + lane (both staged in
            // s_x1); warp 0 folds them in that order
            const unsigned int q = q0 + (unsigned int)it;
            for (int r0 = 0; r0 < G; r0 += 64) {
                const int r = r0 + 32 * warp + lane;
                CdPartial x;
                const bool got = xchg_poll1(xchg + (size_t)(q & 1u) * G * kXchgWords, G, r, q, x);
                if (!got && lane == 0) s_tmo = 1;
                if (got && r < G) s_x1[warp][lane] = x;
                named_bar_sync(2, 64);
                if (s_tmo) { tmo = true; break; }              // uniform over warps 0 and 1
                if (warp == 0) {
                    if (r < G) fold_partial(s_x1[0][lane], r0 == 0, bb, bj, cj, gsum, cnt, err);
                    if (r + 32 < G) fold_partial(s_x1[1][lane], false, bb, bj, cj, gsum, cnt, err);
                }
                if (r0 + 64 < G) named_bar_sync(2, 64);       // s_x1 read before it is restaged
            }
        }
        if (warp == 0) {
            if (ls.have_prev) {
                if (kGrid && it > 0) {
                    // folded above
                } else {
                    for (int r = lane; r < G; r += 64) {       // two loads in flight per lane
                        const bool two = r + 32 < G;
                        // grid mode: the partials of the previous launch (or a restore)
                        const CdPartial x0 = kGrid ? ldcg_partial(gpart + r) : *cluster.map_shared_rank(&spart[pin], r);
                        CdPartial x1;
                        if (two)
                            x1 = kGrid ? ldcg_partial(gpart + r + 32) : *cluster.map_shared_rank(&spart[pin], r + 32);
                        fold_partial(x0, r == lane, bb, bj, cj, gsum, cnt, err);
                        if (two) fold_partial(x1, false, bb, bj, cj, gsum, cnt, err);
                    }
                }
                warp_combine(bb, bj, cj, gsum, cnt, err);
            }
            if (tmo) {
                if (lane == 0) {
                    set_status(st, kErrTimeout);
                    sel.stop = 1;
                    s_tmo = 1;
                }
            } else if (lane == 0) {
                long long nslots = ls.n_slots;
                double pb = 0.0;
                unsigned long long gp = 0ull;
                if (ls.have_prev) {
                    // recalculated b of the previous coordinate (Eq. recalculate-b) and its gradient
                    pb = fma(ls.pHii, ls.pc, gsum);
                    gp = abs_bits(fma(ls.pmu_g, ls.pc, pb));
                    nslots += cnt[3];
                    const long long pdiag = is_zero(ls.pHii) ? 0 : 1;
                    ls.elements += cnt[0] + pdiag;
                    ls.applied += cnt[1] + pdiag;
                    ls.dropped += cnt[2];
                    ls.inserted += cnt[3];
                    ls.last_column = cnt[0] + pdiag;
                }
                sel.pA = ls.pA; sel.pB = ls.pB; sel.pslot = ls.pslot; sel.pb = pb; sel.pc = ls.pc;
                sel.have_prev = ls.have_prev;
                if (ls.forced) {
                    // a start vector's entry: insert it if absent; its c and b as stored now.  The
                    // previous coordinate's recalculated b is written by the element thread that meets
                    // it in this column; an entry more than a double excitation away has no such
                    // element, so CTA 0 writes it here.
                    if (ls.have_prev && rank == 0 &&
                        __popcll(ls.pA ^ ls.fa) + __popcll(ls.pB ^ ls.fb) > 4)
                        P.table[ls.pslot].bv = pb;
                    // every CTA looks the entry up; the one whose insert wins counts it in its partial
                    bool ins = false;
                    const long long fs = table_find(P, st, ls.fa, ls.fb, true, &ins);
                    s_fins = ins ? 1 : 0;
                    sel.iA = ls.fa; sel.iB = ls.fb; sel.islot = fs;
                    sel.ci = fs >= 0 ? __ldcg(&P.table[fs].c) : 0.0;
                    sel.bi = fs >= 0 ? __ldcg(&P.table[fs].bv) : 0.0;
                    sel.feta = ls.feta;
                    sel.forced = 1;
                    sel.stop = (err != 0) || (fs < 0) || (nslots > P.max_entries);
                } else if (better(gp, ls.pA, ls.pB, bb.g, bb.a, bb.b)) {
                    sel.iA = ls.pA; sel.iB = ls.pB; sel.islot = ls.pslot; sel.bi = pb; sel.ci = ls.pc;
                    sel.forced = 0;
                    sel.stop = (err != 0) || (nslots > P.max_entries);
                } else {
                    sel.iA = bb.a; sel.iB = bb.b; sel.islot = bb.slot; sel.bi = bj; sel.ci = cj;
                    sel.forced = 0;
                    sel.stop = (err != 0) || (nslots > P.max_entries) || (bb.slot < 0);
                }
                if (nslots > P.max_entries) set_status(st, kErrTableFull);
                ls.n_slots = nslots;
            }
        }
        }
        __syncthreads();
        if (sel.stop) break;                          // identical in every CTA of the cluster
        const unsigned long long iA = sel.iA, iB = sel.iB;
        const bool have_prev = sel.have_prev != 0;
        const unsigned long long pA = sel.pA, pB = sel.pB;

        // ---- lists (every warp) ----
        ColLists &L = Lw[warp];
        for (int t = lane; t < P.N; t += 32) {
            int ra = __popcll(iA & low_mask(t)), rb = __popcll(iB & low_mask(t));
            if ((iA >> t) & 1ull) L.occA[ra] = (unsigned char)t; else L.virA[t - ra] = (unsigned char)t;
            if ((iB >> t) & 1ull) L.occB[rb] = (unsigned char)t; else L.virB[t - rb] = (unsigned char)t;
        }
        __syncwarp();
        Elem el[kE];
        unsigned long long hAc = 0ull, hBc = 0ull;
        if (warp == 0) {
            // ---- control warp: H_ii and the step size (appendix) ----
            const double Hii = diag_pairs_warp(P, L, sHd, sJ, sK, sPairs, lay.npairs);
            if (lane == 0) {
                const double bi = sel.bi, ci = sel.ci;
                double eta;
                if (sel.forced) {
                    eta = sel.feta;
                } else {
                    const double mu0 = ls.pmu_g;          // c.c within 2 ulp (the double-double value runs behind)
                    eta = line_search(4.0 * bi + 4.0 * mu0 * ci, 2.0 * Hii + 4.0 * ci * ci + 2.0 * mu0, 4.0 * ci);
                }
                sel.eta = eta;
                sel.mu_g = ls.mu.hi + fma(2.0 * eta, ci, eta * eta);
                sel.bad = ((__double_as_longlong(eta) >> 52) & 0x7ff) == 0x7ff;   // not finite
                s_hii = Hii;
            }
#pragma unroll
            for (int k = 0; k < kE; ++k) el[k].state = 0;
        } else {
            // ---- element warps: term loads of this CTA's singles (from the lists alone), the
            // column's single-excitation tables, decode, first probes, values ----
            const int u = tid - 32;
            constexpr int kU = kCdThreads - 32;
            constexpr int kR = 2;
            double tv[kR] = {0.0, 0.0};
            if (tb > 0) {                              // uniform in the CTA; nterms >= 1 then
#pragma unroll
                for (int r = 0; r < kR; ++r)
                    tv[r] = __ldg(single_term_ptr(P, L, rank, G, nocc, nsing, min(u + r * kU, nterms - 1)));
            }
            build_singles(P, L, iA, iB, tabA, tabB, tid - 32, kCdThreads - 32);
            asm volatile("bar.sync 1, %0;" ::"r"(kCdThreads - 32) : "memory");
            hAc = hash_alpha(iA);
            hBc = hash_beta(iB);
#pragma unroll
            for (int k = 0; k < kE; ++k)
                issue_elem(P, L, tabA, tabB, iA, iB, hAc, hBc, e0 + k * stride, nh, have_prev, pA, pB, el[k]);
            // this thread's singles that the term table covers (first round: block (warp - 1) + W' k)
            bool ts[kE];
#pragma unroll
            for (int k = 0; k < kE; ++k) ts[k] = el[k].state != 0 && el[k].ix.kind <= 1 && (warp - 1) + Wp * k < tb;
#pragma unroll
            for (int k = 0; k < kE; ++k)
                if (el[k].state != 0 && !ts[k]) el[k].H = element_value(P, L, el[k].ix);
            if (tb > 0) {                              // uniform in the CTA
#pragma unroll
                for (int r = 0; r < kR; ++r)
                    if (u + r * kU < nterms) sTerm[u + r * kU] = tv[r];
                for (int base = u + kR * kU; base < nterms; base += kR * kU) {
#pragma unroll
                    for (int r = 0; r < kR; ++r)
                        tv[r] = __ldg(single_term_ptr(P, L, rank, G, nocc, nsing, min(base + r * kU, nterms - 1)));
#pragma unroll
                    for (int r = 0; r < kR; ++r)
                        if (base + r * kU < nterms) sTerm[base + r * kU] = tv[r];
                }
                asm volatile("bar.sync 1, %0;" ::"r"(kCdThreads - 32) : "memory");
#pragma unroll
                for (int k = 0; k < kE; ++k)
                    if (ts[k]) {
                        const int ls = ((warp - 1) + Wp * k) * 32 + lane;
                        el[k].H = single_sum(sTerm + ls * (nocc + 1), nocc, el[k].ix.sgn);
                    }
            }
        }
        __syncthreads();
        const double eta = sel.eta;
        const double mu = sel.mu_g;
        const unsigned long long tau_bits = abs_bits(P.tau);
        const long long pslot = sel.pslot;
        const double pb = sel.pb, pc = sel.pc;
        const bool bad = sel.bad != 0;

        // ---- apply: b_j += eta H_ji with compression, gather, candidates ----
        Best best{0ull, ~0ull, ~0ull, -1};
        double bbest = 0.0, cbest = 0.0, gather = 0.0;
        int cnt[4] = {0, 0, 0, 0};                     // elements, applied, dropped, inserted
        int err = 0;
        for (long long eb = e0; !bad && eb < nh;) {
#pragma unroll
            for (int k = 0; k < kE; ++k) resolve_elem(P, st, el[k], &err);
#pragma unroll
            for (int k = 0; k < kE; ++k) {
                Elem &x = el[k];
                if (x.state == 0) continue;
                const double H = x.H;
                const double v = eta * H;
                const bool big = abs_bits(v) >= tau_bits;
                double cj, bn;
                long long sj;
                if (x.state == 3) {                       // the previous coordinate: c and b known
                    cj = pc;
                    sj = pslot;
                    if (is_zero(H)) { P.table[sj].bv = pb; continue; }
                    ++cnt[0];
                    if (!(!is_zero(cj) || big)) { P.table[sj].bv = pb; ++cnt[2]; continue; }
                    bn = pb + v;
                } else if (x.state == 1) {
                    cj = x.cb0.x;
                    sj = x.pos;
                    ++cnt[0];
                    if (!(!is_zero(cj) || big)) { ++cnt[2]; continue; }
                    bn = x.cb0.y + v;
                } else {                                  // absent
                    ++cnt[0];
                    if (!big) { ++cnt[2]; continue; }
                    sj = claim_slot(P, st, x.ka, x.kb, x.pos, &err);
                    if (sj < 0) continue;
                    cj = 0.0;
                    bn = v;
                    ++cnt[3];
                }
                ++cnt[1];
                P.table[sj].bv = bn;
                unsigned long long gb;
                if (!is_zero(cj)) {
                    gather = fma(H, cj, gather);
                    gb = abs_bits(fma(mu, cj, bn));
                } else {
                    gb = abs_bits(bn);
                }
                if (better(gb, x.ka, x.kb, best.g, best.a, best.b)) {
                    best = Best{gb, x.ka, x.kb, sj};
                    bbest = bn;
                    cbest = cj;
                }
            }
            eb += kE * stride;
            if (eb >= nh) break;
#pragma unroll
            for (int k = 0; k < kE; ++k)
                issue_elem(P, L, tabA, tabB, iA, iB, hAc, hBc, eb + k * stride, nh, have_prev, pA, pB, el[k]);
#pragma unroll
            for (int k = 0; k < kE; ++k)
                if (el[k].state != 0) el[k].H = element_value(P, L, el[k].ix);
        }

        // ---- CTA partial into this CTA's shared memory ----
        if (warp != 0) warp_combine(best, bbest, cbest, gather, cnt, err);   // warp 0 holds no elements
        if (lane == 0) {
            r_best[warp] = best;
            r_bc[warp][0] = bbest;
            r_bc[warp][1] = cbest;
            r_bc[warp][2] = gather;
            for (int k = 0; k < 4; ++k) r_cnt[k][warp] = cnt[k];
            if (err) atomicOr(&s_err, 1);
        }
        __syncthreads();
        if (warp == 1 && lane < 2) {
            // beside the control warp's combine, on another scheduler and with the FP64 pipe of the
            // element warps idle: lane 0: mu += 2 eta c_i + eta^2; lane 1: alpha += 2 eta b_i +
            // eta^2 H_ii (double-double); read by the next iteration after the barrier
            const dd x0 = lane == 0 ? ls.mu : ls.alpha;
            const double y1 = lane == 0 ? sel.ci : sel.bi;
            const double y2 = lane == 0 ? 1.0 : s_hii;
            const dd t = dd_add_fast(dd_two_prod(2.0 * eta, y1), dd_mul_d(dd_two_prod(eta, eta), y2));
            const dd r = dd_add_fast(x0, t);
            if (lane == 0) ls.mu = r; else ls.alpha = r;
        }
        if (warp == 0) {
            const bool have = lane < kCdWarps;
            Best b = have ? r_best[lane] : Best{0ull, ~0ull, ~0ull, -1};
            double bj = have ? r_bc[lane][0] : 0.0, cj = have ? r_bc[lane][1] : 0.0;
            double gs = have ? r_bc[lane][2] : 0.0;
            int c4[4] = {have ? r_cnt[0][lane] : 0, have ? r_cnt[1][lane] : 0, have ? r_cnt[2][lane] : 0,
                         have ? r_cnt[3][lane] : 0};
            int e2 = 0;
            warp_combine(b, bj, cj, gs, c4, e2);
            if (lane == 0) {
                CdPartial pp;
                pp.gbits = b.g; pp.ka = b.a; pp.kb = b.b; pp.slot = b.slot;
                pp.bj = bj; pp.cj = cj; pp.gather = gs;
                pp.elements = c4[0]; pp.applied = c4[1]; pp.dropped = c4[2]; pp.inserted = c4[3] + s_fins;
                s_fins = 0;
                pp.err = s_err | (bad ? 1 : 0);
                if (kGrid) spart[0] = pp; else spart[pout] = pp;
                // the coordinate's own slot: c_i += eta, b_i as used (rank 0 writes)
                const double ci = sel.ci, ci_new = ci + sel.eta;
                if (rank == 0 && !bad) {
                    P.table[sel.islot].c = ci_new;
                    P.table[sel.islot].bv = sel.bi;
                }
                if (bad && rank == 0) set_status(st, kErrNonfinite);
            }
            if (kGrid) {
                __syncwarp();
                const unsigned int q = q0 + (unsigned int)it + 1u;
                xchg_publish(xchg + ((size_t)(q & 1u) * G + rank) * kXchgWords, spart[0], q, lane);
            }
            if (lane == 0) {
                const double ci = sel.ci, ci_new = ci + sel.eta;
                ls.pA = sel.iA; ls.pB = sel.iB; ls.pslot = sel.islot;
                ls.pc = ci_new; ls.pHii = s_hii; ls.pmu_g = sel.mu_g; ls.peta = sel.eta;
                if (!sel.forced) {
                    ls.iterations += 1;
                    ls.dx = P.theta * ls.dx + (1.0 - P.theta) * fabs(sel.eta);
                    // (dx >= 0: the bit patterns of non-negative doubles order like their values)
                    const long long dxb = __double_as_longlong(ls.dx), thb = __double_as_longlong(P.dx_threshold);
                    if (thb > 0 && dxb < thb) ls.done = 1;
                }
                const bool z0 = is_zero(ci), z1 = is_zero(ci_new);
                ls.nnz_c += ((z0 && !z1) ? 1 : 0) - ((!z0 && z1) ? 1 : 0);
                ls.forced = 0;
                ls.have_prev = 1;
                s_done = ls.done;
            }
        }
        if (kGrid) {
            ++n_pub;
            __syncthreads();                          // s_done; the partials travel through xchg
        } else if (G == 1) {
            __syncthreads();
        } else {
            cluster.sync();                           // partials and table writes visible cluster-wide
        }
        lastp = pout;
        if (s_done || bad) break;                     // identical in every CTA
    }

    // ---- state for the next launch / the finalisation ----
    if (kGrid && n_pub > 0 && warp == 0 && !s_tmo) {
        // every CTA's last partial published, so no CTA still reads gpart, rec or the buffers of
        // this launch: this CTA's last partial becomes its gpart entry, rank 0 advances the rounds
        const unsigned int q = q0 + n_pub;
        bool fin = true;
        for (int r0 = 0; r0 < G && fin; r0 += 32) {
            CdPartial x;
            fin = xchg_poll1(xchg + (size_t)(q & 1u) * G * kXchgWords, G, r0 + lane, q, x);
        }
        if (lane == 0) {
            if (fin) {
                gpart[rank] = spart[0];
                if (rank == 0) rnd->round = __ldcg(&rnd->round) + n_pub;   // written by rank 0 alone
            } else {
                set_status(st, kErrTimeout);
            }
        }
    }
    if (!kGrid && tid == 0) gpart[rank] = spart[lastp];
    if (tid == 0 && rank == 0) {      // lane 0 of the control warp holds the state
        CdRecord o;
        o.a = ls.pA; o.b = ls.pB; o.slot = ls.pslot;
        o.c_new = ls.pc; o.Hii = ls.pHii; o.eta = ls.peta;
        o.mu = ls.mu; o.alpha = ls.alpha; o.dx = ls.dx; o.mu_g = ls.pmu_g;
        o.energy = dd_div_to_d(ls.alpha, ls.mu);
        o.iterations = ls.iterations; o.nnz_c = ls.nnz_c; o.n_slots = ls.n_slots; o.elements = ls.elements;
        o.applied = ls.applied; o.dropped = ls.dropped; o.inserted = ls.inserted; o.last_column = ls.last_column;
        o.fa = ls.fa; o.fb = ls.fb; o.feta = ls.feta;
        o.forced = ls.forced; o.have_prev = ls.have_prev; o.done = ls.done;
        *rec = o;
    }
}

// kE: element slots a thread keeps in flight; 1 when one round of the CTAs'
// threads covers the column (the smaller loop body is faster), else kCdMaxE.
template <int kE>
__global__ void __launch_bounds__(kCdThreads, 1) k_cd_loop(Problem P, IterState *st, CdRecord *rec,
                                                           CdPartial *gpart, long long n_iter) {
    cd_loop_body<false, kE>(P, st, rec, gpart, nullptr, nullptr, n_iter);
}

// the loop over every CTA of a cooperative launch (see cd_loop_body)
template <int kE>
__global__ void __launch_bounds__(kCdThreads, 1) k_cd_loop_grid(Problem P, IterState *st, CdRecord *rec,
                                                                CdPartial *gpart, unsigned long long *xchg,
                                                                GridRound *rnd, long long n_iter) {
    cd_loop_body<true, kE>(P, st, rec, gpart, xchg, rnd, n_iter);
}

// Many independent problems in one launch: cluster k (blocks k*G .. k*G+G-1)
// runs the loop above on instance k, whose description it first copies into
// shared memory.  Clusters never wait on one another.
__global__ void __launch_bounds__(kCdThreads, 1) k_cd_loop_batch(const CdInstance *inst, int n_inst,
                                                                 long long n_iter) {
    __shared__ Problem sP;
    namespace cg = cooperative_groups;
    const int k = (int)(blockIdx.x / cg::this_cluster().num_blocks());
    if (k >= n_inst) return;                           // uniform in the cluster
    for (int t = threadIdx.x; t < (int)(sizeof(Problem) / 8); t += blockDim.x)
        reinterpret_cast<unsigned long long *>(&sP)[t] = reinterpret_cast<const unsigned long long *>(&inst[k].P)[t];
    __syncthreads();
    cd_loop_body<false, kCdMaxE>(sP, inst[k].st, inst[k].rec, inst[k].part, nullptr, nullptr, n_iter);
}

// After a batch of iterations: write the pending recalculated b_i of the last
// processed coordinate and a host-visible snapshot of the counters.
__device__ __forceinline__ void cd_finalize_body(const Problem &P, IterState *st, const CdRecord *rec,
                                                 const CdPartial *gpart, int G) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const CdRecord R = *rec;
    // the same per-lane fold (CTAs lane, lane + 32, ...) and tree as the loop's choice
    double gsum = 0.0;
    long long cnt[4] = {0, 0, 0, 0};
    if (R.have_prev)
        for (int r = lane; r < G; r += 32) {
            const CdPartial x = gpart[r];
            gsum = (r == lane) ? x.gather : gsum + x.gather;
            cnt[0] += x.elements; cnt[1] += x.applied; cnt[2] += x.dropped; cnt[3] += x.inserted;
        }
    for (int off = 16; off > 0; off >>= 1) {
        gsum += __shfl_down_sync(0xffffffffu, gsum, off);
        for (int k = 0; k < 4; ++k) cnt[k] += __shfl_down_sync(0xffffffffu, cnt[k], off);
    }
    if (lane != 0) return;
    const long long pdiag = (R.have_prev && R.Hii != 0.0) ? 1 : 0;
    if (R.have_prev && st->status == 0) P.table[R.slot].bv = fma(R.Hii, R.c_new, gsum);
    st->iterations = R.iterations;
    st->nnz_c = R.nnz_c;
    st->n_slots = R.n_slots + cnt[3];
    st->elements = R.elements + cnt[0] + pdiag;
    st->applied = R.applied + cnt[1] + pdiag;
    st->dropped = R.dropped + cnt[2];
    st->inserted = R.inserted + cnt[3];
    st->last_column = R.have_prev ? cnt[0] + pdiag : 0;
    st->mu = R.mu;
    st->alpha = R.alpha;
    st->dx = R.dx;
    st->energy = R.energy;
    st->last_eta = R.eta;
    st->last_a = R.a;
    st->last_b = R.b;
    st->done = R.done;
    if (st->n_slots > P.max_entries) set_status(st, kErrTableFull);
}

__global__ void k_cd_finalize(Problem P, IterState *st, const CdRecord *rec, const CdPartial *gpart, int G) {
    cd_finalize_body(P, st, rec, gpart, G);
}

// one warp per instance
__global__ void k_cd_finalize_batch(const CdInstance *inst, int n_inst, int G) {
    const int k = blockIdx.x;
    if (k >= n_inst) return;
    cd_finalize_body(inst[k].P, inst[k].st, inst[k].rec, inst[k].part, G);
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
            keys[2 * pos + 1] = sl.b & kKeyMaskB;
            if (c) c[pos] = sl.c * s;
            if (b) b[pos] = sl.bv * s;
        }
    }
}

// ---------------------------------------------------------------------------
// Checkpoint / restore
// ---------------------------------------------------------------------------
// Every stored entry as stored (c, b divided by the scale for m > 1); flags
// bit 0: the entry is marked as a candidate of the next block selection.
__global__ void k_ckpt_export(Problem P, unsigned long long *keys, double *c, double *b, unsigned char *flags,
                              long long cap, unsigned long long *counter) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.capacity;
         i += (long long)gridDim.x * blockDim.x) {
        const Slot sl = P.table[i];
        if (sl.a == 0ull && sl.b == 0ull) continue;
        const unsigned long long pos = atomicAdd(counter, 1ull);
        if ((long long)pos >= cap) continue;
        keys[2 * pos] = sl.a;
        keys[2 * pos + 1] = sl.b & kKeyMaskB;
        c[pos] = sl.c;
        b[pos] = sl.bv;
        flags[pos] = (P.mark ? mark_test(P, i) : (sl.b & kMarkB) != 0ull) ? 1 : 0;
    }
}

// The pending partials of the last m = 1 column folded by one warp exactly as
// the next step's choice folds them (lane l takes CTAs l, l + 32, ...; then
// the warp combine); lane 0 writes the result.
__global__ void k_ckpt_fold(const CdPartial *gpart, int G, CdPartial *out) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    Best bb{0ull, ~0ull, ~0ull, -1};
    double bj = 0.0, cj = 0.0, gsum = 0.0;
    int cnt[4] = {0, 0, 0, 0};
    int err = 0;
    for (int r = lane; r < G; r += 32) fold_partial(gpart[r], r == lane, bb, bj, cj, gsum, cnt, err);
    warp_combine(bb, bj, cj, gsum, cnt, err);
    if (lane == 0) {
        CdPartial x;
        x.gather = gsum; x.gbits = bb.g; x.ka = bb.a; x.kb = bb.b; x.slot = bb.slot;
        x.bj = bj; x.cj = cj;
        x.elements = cnt[0]; x.applied = cnt[1]; x.dropped = cnt[2]; x.inserted = cnt[3];
        x.err = err;
        *out = x;
    }
}

// Re-insert checkpoint rows (the table is empty): c and b as stored; rows with
// flag bit 0 are marked and listed as candidates (m > 1).  A key found instead
// of inserted (a repeated row) is a consistency error.
__global__ void k_ckpt_import(Problem P, IterState *st, const unsigned long long *keys, const double *c,
                              const double *b, const unsigned char *flags, long long n, long long *cand,
                              int *n_cand, long long cap_cand) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        bool ins = false;
        const long long s = table_find(P, st, keys[2 * i], keys[2 * i + 1], true, &ins);
        if (s < 0) continue;                                  // table full: status set
        if (!ins) { set_status(st, kErrInternal); continue; }
        P.table[s].c = c[i];
        P.table[s].bv = b[i];
        if (c[i] != 0.0) cnz_set(P, keys[2 * i], keys[2 * i + 1]);
        if (flags && (flags[i] & 1) && cand) {
            if (P.mark) mark_set(P, s);
            else P.table[s].b = keys[2 * i + 1] | kMarkB;
            const int pos = atomicAdd(n_cand, 1);
            if (pos < cap_cand) cand[pos] = s;
            else set_status(st, kErrInternal);
        }
    }
}

// m = 1 restore after the rows are in: the record (slots looked up by key) and
// the pending partials, the folded one at CTA 0 and empty ones elsewhere.
__global__ void k_ckpt_restore_m1(Problem P, IterState *st, CdRecord *rec, CdPartial *gpart, int G, CdRecord r,
                                  CdPartial folded) {
    if (threadIdx.x == 0) {
        bool ins = false;
        if (r.have_prev) {
            r.slot = table_find(P, st, r.a, r.b, false, &ins);
            if (r.slot < 0) { set_status(st, kErrInternal); r.slot = 0; }
        }
        if (folded.slot >= 0) {
            folded.slot = table_find(P, st, folded.ka, folded.kb, false, &ins);
            if (folded.slot < 0) set_status(st, kErrInternal);
        }
        *rec = r;
        gpart[0] = folded;
    }
    for (int k = 1 + threadIdx.x; k < G; k += blockDim.x) {
        CdPartial e;
        e.gather = 0.0; e.gbits = 0ull; e.ka = ~0ull; e.kb = ~0ull; e.slot = -1; e.bj = 0.0; e.cj = 0.0;
        e.elements = 0; e.applied = 0; e.dropped = 0; e.inserted = 0; e.err = 0;
        gpart[k] = e;
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
            s_a = sl.a; s_b = sl.b & kKeyMaskB; s_ci = sl.c;
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
// 4-fold form (complex orbitals with real integrals): (pq|rs) = (rs|pq) = (qp|sr)
__global__ void k_validate_g4(const double *g, int N, double tol, int *status) {
    const long long n4 = (long long)N * N * N * N;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t % N), r = (int)((t / N) % N), q = (int)((t / N / N) % N), p = (int)(t / N / N / N);
        const double x = g[t];
        const double y1 = g[(((long long)r * N + s) * N + p) * N + q], y2 = g[(((long long)q * N + p) * N + s) * N + r];
        if (!isfinite(x)) { atomicCAS(status, 0, kErrNonfinite); continue; }
        if (fabs(x - y1) > tol * fmax(1.0, fabs(y1)) || fabs(x - y2) > tol * fmax(1.0, fabs(y2)))
            atomicCAS(status, 0, kErrArg);
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

// Single-excitation term tables (Eq. entry, singles): for the excitation i -> a
// an occupied orbital k of the same spin contributes (ia|kk) - (ik|ka) and one
// of the other spin (ia|kk); W3 and V3 hold these per (i, a, k), so that the
// terms of one single lie in two rows of N doubles.
__global__ void k_w3v3(const double *g, int N, double *W3, double *V3) {
    const long long n3 = (long long)N * N * N;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t % N), a = (int)((t / N) % N), i = (int)(t / N / N);
        W3[t] = gi(g, N, i, a, k, k) - gi(g, N, i, k, k, a);
        V3[t] = gi(g, N, i, a, k, k);
    }
}

// Insert the start determinant and write the record that makes the next
// iteration the initialisation: c = e_ref reached from c = 0 with eta = 1,
// so mu = 1 and alpha = H_ref,ref.
// The record of a fresh start: nothing processed yet, the next step forced onto
// {A, B} with step eta (from c = 0: c = eta e_{A,B}, the start vector of r4).
__global__ void k_init_state(IterState *st, CdRecord *rec, unsigned long long A, unsigned long long B, double eta) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    CdRecord r;
    r.a = 0ull; r.b = 0ull; r.slot = 0;
    r.c_new = 0.0; r.Hii = 0.0; r.eta = 0.0;
    r.mu = dd_from(0.0); r.alpha = dd_from(0.0);
    r.dx = 0.0; r.energy = 0.0;
    r.iterations = 0; r.nnz_c = 0; r.n_slots = 0; r.elements = 0; r.applied = 0; r.dropped = 0;
    r.inserted = 0; r.last_column = 0;
    r.fa = A; r.fb = B; r.feta = eta;
    r.forced = 1;
    r.have_prev = 0;
    r.done = 0;
    r.mu_g = 0.0;
    rec[0] = r;
    st->last_parity = 0;
    st->scale = dd_from(1.0);
}

// The next step forced onto start-vector entry k (keys 2k, 2k + 1; step c[k]).
__global__ void k_force_next(CdRecord *rec, const unsigned long long *keys, const double *c, long long k) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    rec->fa = keys[2 * k];
    rec->fb = keys[2 * k + 1];
    rec->feta = c[k];
    rec->forced = 1;
}

// ---------------------------------------------------------------------------
// Launch wrappers (host)
// ---------------------------------------------------------------------------
// One element slot per thread suffices when the G CTAs' element threads cover
// the column in one round.
static bool cd_one_round(const Problem &P, int G) {
    const long long nh = P.doubles_vanish ? P.seg[2] : P.seg[5];
    return (long long)G * (kCdWarps - 1) * 32 >= nh - 1;
}

cudaError_t launch_cd_loop(const Problem &P, IterState *st, CdRecord *rec, CdPartial *part, int cluster,
                           long long n_iter, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(kCdThreads);
    cfg.dynamicSmemBytes = cd_dynamic_smem(P);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cd_one_round(P, cluster)) return cudaLaunchKernelEx(&cfg, k_cd_loop<1>, P, st, rec, part, n_iter);
    return cudaLaunchKernelEx(&cfg, k_cd_loop<kCdMaxE>, P, st, rec, part, n_iter);
}

cudaError_t launch_cd_loop_batch(const CdInstance *inst, int n_inst, int cluster, size_t smem, long long n_iter,
                                 cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_cd_loop_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(k_cd_loop_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, kCdMaxDynSmem);
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_inst * cluster));
    cfg.blockDim = dim3(kCdThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_cd_loop_batch, inst, n_inst, n_iter);
}

cudaError_t launch_cd_finalize_batch(const CdInstance *inst, int n_inst, int cluster, cudaStream_t s) {
    k_cd_finalize_batch<<<n_inst, 32, 0, s>>>(inst, n_inst, cluster);
    return cudaGetLastError();
}

// The grid-wide loop: G co-resident CTAs (cooperative launch); gpart
// holds G partials, xchg 2 G kXchgWords zero-initialised words, rnd a
// zero-initialised GridRound (both kept between launches).
cudaError_t launch_cd_loop_grid(const Problem &P, IterState *st, CdRecord *rec, CdPartial *gpart,
                                unsigned long long *xchg, GridRound *rnd, int G, long long n_iter, cudaStream_t s) {
    if (G < 1) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kCdThreads);
    cfg.dynamicSmemBytes = cd_dynamic_smem(P);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cd_one_round(P, G)) return cudaLaunchKernelEx(&cfg, k_cd_loop_grid<1>, P, st, rec, gpart, xchg, rnd, n_iter);
    return cudaLaunchKernelEx(&cfg, k_cd_loop_grid<kCdMaxE>, P, st, rec, gpart, xchg, rnd, n_iter);
}

// The largest CTA count of the grid-wide loop that can be co-resident (0 if none).
int cd_max_grid(size_t smem) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_cd_loop_grid<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCdMaxDynSmem);
        cudaFuncSetAttribute(k_cd_loop_grid<kCdMaxE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCdMaxDynSmem);
        attr_set = true;
    }
    int dev = 0, sms = 0, per = 0, per1 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cd_loop_grid<kCdMaxE>, kCdThreads, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_cd_loop_grid<1>, kCdThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms * std::min(per, per1);
}

size_t cd_dynamic_smem(const Problem &P) { return cd_smem_layout(P).bytes; }

// Smallest power-of-two cluster size >= want (at most 16) that can be resident.
int cd_pick_cluster(int want, size_t smem) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_cd_loop<1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(k_cd_loop<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCdMaxDynSmem);
        cudaFuncSetAttribute(k_cd_loop<kCdMaxE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaFuncSetAttribute(k_cd_loop<kCdMaxE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCdMaxDynSmem);
        attr_set = true;
    }
    int c = 1;
    while (c < want && c * 2 <= kCdMaxCluster) c *= 2;
    for (; c > 1; c /= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kCdThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        int n1 = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_cd_loop<kCdMaxE>, &cfg) == cudaSuccess && n >= 1 &&
            cudaOccupancyMaxActiveClusters(&n1, k_cd_loop<1>, &cfg) == cudaSuccess && n1 >= 1)
            return c;
        cudaGetLastError();
    }
    return 1;
}

cudaError_t launch_cd_finalize(const Problem &P, IterState *st, CdRecord *rec, CdPartial *part, int cluster,
                               cudaStream_t s) {
    k_cd_finalize<<<1, 32, 0, s>>>(P, st, rec, part, cluster);
    return cudaGetLastError();
}

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

cudaError_t launch_ckpt_export(const Problem &P, unsigned long long *keys, double *c, double *b, unsigned char *flags,
                               long long cap, unsigned long long *counter, cudaStream_t s) {
    long long grid = (P.capacity + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    k_ckpt_export<<<(int)grid, 256, 0, s>>>(P, keys, c, b, flags, cap, counter);
    return cudaGetLastError();
}

cudaError_t launch_ckpt_fold(const CdPartial *gpart, int G, CdPartial *out, cudaStream_t s) {
    k_ckpt_fold<<<1, 32, 0, s>>>(gpart, G, out);
    return cudaGetLastError();
}

cudaError_t launch_ckpt_import(const Problem &P, IterState *st, const unsigned long long *keys, const double *c,
                               const double *b, const unsigned char *flags, long long n, long long *cand, int *n_cand,
                               long long cap_cand, cudaStream_t s) {
    long long grid = (n + 255) / 256;
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_ckpt_import<<<(int)grid, 256, 0, s>>>(P, st, keys, c, b, flags, n, cand, n_cand, cap_cand);
    return cudaGetLastError();
}

cudaError_t launch_ckpt_restore_m1(const Problem &P, IterState *st, CdRecord *rec, CdPartial *gpart, int G,
                                   const CdRecord &r, const CdPartial &folded, cudaStream_t s) {
    k_ckpt_restore_m1<<<1, 256, 0, s>>>(P, st, rec, gpart, G, r, folded);
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

cudaError_t launch_setup(double *h, double *g, int N, double *J, double *K, double *W3, double *V3, int *status,
                         int *has_doubles, int sym4, cudaStream_t s) {
    long long n4 = (long long)N * N * N * N;
    int grid = (int)((n4 + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_validate_h<<<4, 256, 0, s>>>(h, N, 1e-12, status);
    if (sym4) {
        k_validate_g4<<<grid, 256, 0, s>>>(g, N, 1e-12, status);
    } else {
        k_validate_g<<<grid, 256, 0, s>>>(g, N, 1e-12, status);
    }
    k_symmetrize_h<<<4, 256, 0, s>>>(h, N);
    if (!sym4) k_canonicalize_g<<<grid, 256, 0, s>>>(g, N);
    k_jk<<<grid, 256, 0, s>>>(g, N, J, K, has_doubles);
    const long long n3 = (long long)N * N * N;
    k_w3v3<<<(int)std::min<long long>((n3 + 255) / 256, 1024), 256, 0, s>>>(g, N, W3, V3);
    return cudaGetLastError();
}

cudaError_t launch_init_state(IterState *st, CdRecord *rec, unsigned long long A, unsigned long long B, double eta,
                              cudaStream_t s) {
    k_init_state<<<1, 32, 0, s>>>(st, rec, A, B, eta);
    return cudaGetLastError();
}

cudaError_t launch_force_next(CdRecord *rec, const unsigned long long *keys, const double *c, long long k,
                              cudaStream_t s) {
    k_force_next<<<1, 32, 0, s>>>(rec, keys, c, k);
    return cudaGetLastError();
}

}  // namespace cdfci
