// Library-internal definitions shared by the CUDA translation units of libcdfci.
//
// Device data layout (one solver handle):
//   table      : 2^k slots of 32 bytes {uint64 A, uint64 B, double c, double b}
//                (one DRAM sector per determinant: key, coefficient, b = Hc).
//                Empty slot: A = B = 0 (no valid determinant has both words 0).
//                c and b are stored divided by a global scale s (c_true = s*c),
//                so that the multicoordinate update c <- gamma c is O(1).
//   h, g       : FP64 integrals, g in full N^4 chemists' order (L2-resident).
//   J, K       : N*N tables (pp|qq) and (pq|qp) for diagonal elements.
//   pair tables: the (o1 < o2) index pairs of occupied/virtual lists, so a flat
//                excitation index decodes without search.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cdfci {

constexpr int kMaxN = 63;
constexpr int kMaxPairs = 63 * 62 / 2;     // C(63, 2)
constexpr int kStatusOk = 0;

// error codes mirror include/cdfci.h
constexpr int kErrArg = -1, kErrNonfinite = -2, kErrTableFull = -3, kErrTimeout = -4,
              kErrNotNegative = -9;

struct __align__(32) Slot {
    unsigned long long a, b;
    double c, bv;
};

// ---------------------------------------------------------------------------
// Double-double arithmetic: the error-free transformations TwoSum (Knuth,
// TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971) and TwoProduct via a fused
// multiply-add; a value is the unevaluated sum hi + lo.
// ---------------------------------------------------------------------------
struct dd {
    double hi, lo;
};

__host__ __device__ __forceinline__ dd dd_two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__host__ __device__ __forceinline__ dd dd_fast_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    return {s, e};
}
__host__ __device__ __forceinline__ dd dd_two_prod(double a, double b) {
    double p = a * b;
    double e = fma(a, b, -p);
    return {p, e};
}
__host__ __device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    dd t = dd_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = dd_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return dd_fast_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ dd dd_mul_d(dd a, double b) {
    dd p = dd_two_prod(a.hi, b);
    p.lo = fma(a.lo, b, p.lo);
    return dd_fast_two_sum(p.hi, p.lo);
}
__host__ __device__ __forceinline__ dd dd_mul(dd a, dd b) {
    dd p = dd_two_prod(a.hi, b.hi);
    p.lo = fma(a.hi, b.lo, fma(a.lo, b.hi, p.lo));
    return dd_fast_two_sum(p.hi, p.lo);
}
__host__ __device__ __forceinline__ double dd_div_to_d(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_add(a, dd_mul_d(b, -q1));
    double q2 = r.hi / b.hi;
    return q1 + q2;
}
__host__ __device__ __forceinline__ dd dd_from(double x) { return {x, 0.0}; }

// ---------------------------------------------------------------------------
// Per-handle device state of the iteration (one copy in device memory).
// ---------------------------------------------------------------------------
struct IterState {
    // coordinate chosen for the next update (written by the tail of a launch)
    unsigned long long sel_a, sel_b;
    long long sel_slot;
    int forced_eta_one;        // 1 = initialisation: c = e_ref (eta = 1 from c = 0)
    int done;                  // 1 = converged (dx < threshold); launches return at once
    int status;                // first error code (sticky)
    unsigned int arrive;       // arrival ticket of the fused column kernel
    // scalars (double-double), global scale, damped accumulator
    dd mu, alpha;
    dd scale;                  // s: c_true = s * c_stored
    double dx;
    double energy;
    long long iterations;
    // record of the last update
    double last_eta;
    unsigned long long last_a, last_b;
    // counters
    long long nnz_c, n_slots, last_column, elements, applied, dropped, inserted;
};

// per-CTA partial results of the fused m = 1 column kernel
struct __align__(16) CdPartial {
    double gather;                 // sum_j H_ji c_j over this CTA's elements
    unsigned long long gbits;      // |gradient| bits of this CTA's best candidate
    unsigned long long ka, kb;     // its key
    long long slot;                // its slot
    int elements, applied, dropped, inserted;
};

// Everything a kernel needs about the problem and the table.
struct Problem {
    int N, na, nb, va, vb;
    int ca2, cb2, cva2, cvb2;      // C(na,2), C(nb,2), C(va,2), C(vb,2)
    long long seg[6];              // flat column segments: 0 diag | sa | sb | daa | dbb | dab | end=seg[5]
    long long nh;                  // enumeration length (= seg[5])
    int doubles_vanish;            // all (pq|rs) with p != q and r != s are zero (e.g. Hubbard)
    const double *h, *g, *J, *K;
    const unsigned short *pair_oa, *pair_ob, *pair_va, *pair_vb;   // (i | j << 8), i < j
    Slot *table;
    unsigned long long mask;       // capacity - 1
    long long capacity;
    long long max_entries;         // floor(max_load * capacity)
    int max_probe;
    double tau;
    double theta, dx_threshold;
};

// ---------------------------------------------------------------------------
// Bits and hashing
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long low_mask(int bit) {   // bits [0, bit)
    return bit <= 0 ? 0ull : (bit >= 64 ? ~0ull : ((1ull << bit) - 1ull));
}
__device__ __forceinline__ unsigned long long between_mask(int x, int y) {   // strictly between
    int lo = x < y ? x : y, hi = x < y ? y : x;
    return low_mask(hi) & ~low_mask(lo + 1);
}
__device__ __forceinline__ double parity_sign(unsigned long long x) {
    return (__popcll(x) & 1) ? -1.0 : 1.0;
}
// SplitMix64 output finalizer (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ unsigned long long key_hash(unsigned long long a, unsigned long long b) {
    return mix64(a ^ mix64(b ^ 0x9e3779b97f4a7c15ull));
}
// key order for tie-breaks: unsigned 128-bit (B << 64) | A
__device__ __forceinline__ bool key_less(unsigned long long a1, unsigned long long b1,
                                         unsigned long long a2, unsigned long long b2) {
    return b1 != b2 ? b1 < b2 : a1 < a2;
}

// 16-byte compare-and-swap (PTX atom.cas.b128, sm_90 and later)
__device__ __forceinline__ void cas128(unsigned long long *p, unsigned long long clo, unsigned long long chi,
                                       unsigned long long vlo, unsigned long long vhi,
                                       unsigned long long &olo, unsigned long long &ohi) {
    asm volatile(
        "{\n\t.reg .b128 d, c, v;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(olo), "=l"(ohi)
        : "l"(clo), "l"(chi), "l"(vlo), "l"(vhi), "l"(p)
        : "memory");
}

__device__ __forceinline__ void set_status(IterState *st, int code) {
    atomicCAS(&st->status, 0, code);
}

// Look up key {a, b}; insert it if absent and `insert` is set.  Returns the
// slot index, or -1 (absent, not inserted), or -2 (probe limit / timeout;
// status set).  *inserted is set when this call created the entry.
__device__ __forceinline__ long long table_find(const Problem &P, IterState *st, unsigned long long a,
                                                unsigned long long b, bool insert, bool *inserted) {
    unsigned long long pos = key_hash(a, b) & P.mask;
    const bool both_nonzero = (P.na > 0) && (P.nb > 0);
    for (int probe = 0; probe < P.max_probe; ++probe) {
        Slot *s = P.table + pos;
        unsigned long long ka = __ldcg(&s->a), kb = __ldcg(&s->b);
        // a half-written key can only be seen while another thread inserts it
        int spins = 0;
        while (both_nonzero && ((ka == 0ull) != (kb == 0ull))) {
            if (++spins > (1 << 20)) { set_status(st, kErrTimeout); return -2; }
            ka = __ldcg(&s->a);
            kb = __ldcg(&s->b);
        }
        if (ka == a && kb == b) return (long long)pos;
        if (ka == 0ull && kb == 0ull) {
            if (!insert) return -1;
            unsigned long long oa, ob;
            cas128(&s->a, 0ull, 0ull, a, b, oa, ob);
            if (oa == 0ull && ob == 0ull) { *inserted = true; return (long long)pos; }
            if (oa == a && ob == b) return (long long)pos;
        }
        pos = (pos + 1) & P.mask;
    }
    set_status(st, kErrTableFull);
    return -2;
}

// ---------------------------------------------------------------------------
// Column decoding.  Per column the CTA holds the occupied / virtual orbital
// lists of both spins in shared memory.
// ---------------------------------------------------------------------------
struct ColLists {
    unsigned char occA[64], virA[64], occB[64], virB[64];
};

// Fill the lists for key {A, B}; all threads of the block take part.
__device__ __forceinline__ void build_lists(ColLists &L, int N, unsigned long long A, unsigned long long B) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        int ra = __popcll(A & low_mask(t)), rb = __popcll(B & low_mask(t));
        if ((A >> t) & 1ull) L.occA[ra] = (unsigned char)t; else L.virA[t - ra] = (unsigned char)t;
        if ((B >> t) & 1ull) L.occB[rb] = (unsigned char)t; else L.virB[t - rb] = (unsigned char)t;
    }
}

__device__ __forceinline__ double gi(const double *g, int N, int p, int q, int r, int s) {
    return __ldg(g + (((size_t)p * N + q) * N + r) * N + s);
}

// One element of the column of {A, B}: flat index e in [1, nh).  Returns the
// value H_{D',D} (0.0 when the Slater-Condon element vanishes) and the key D'.
// Singles (i -> a, same spin): h_ia + sum_{k in occ same spin} [(ia|kk) - (ik|ka)]
// + sum_{k in occ other spin} (ia|kk), times the sign of the bits strictly
// between i and a.  Same-spin doubles (i<j -> a<b, applied as i->a then
// j->b): sign1 * sign2 * [(ia|jb) - (ib|ja)].  Opposite-spin doubles
// (i->a alpha, j->b beta): signA * signB * (ia|jb).
__device__ __forceinline__ double column_element(const Problem &P, const ColLists &L, unsigned long long A,
                                                 unsigned long long B, long long e, unsigned long long &oa,
                                                 unsigned long long &ob) {
    const int N = P.N;
    const double *g = P.g;
    if (e < P.seg[2]) {                       // singles
        bool alpha = e < P.seg[1];
        long long idx = e - (alpha ? P.seg[0] : P.seg[1]);
        int v = alpha ? P.va : P.vb;
        int o = (int)(idx / v), w = (int)(idx - (long long)o * v);
        int i = alpha ? L.occA[o] : L.occB[o];
        int a = alpha ? L.virA[w] : L.virB[w];
        unsigned long long X = alpha ? A : B;
        double x = __ldg(P.h + i * N + a);
        const unsigned char *os = alpha ? L.occA : L.occB;
        const unsigned char *oo = alpha ? L.occB : L.occA;
        int ns = alpha ? P.na : P.nb, no = alpha ? P.nb : P.na;
        for (int k = 0; k < ns; ++k) {
            int kk = os[k];
            x += gi(g, N, i, a, kk, kk) - gi(g, N, i, kk, kk, a);
        }
        for (int k = 0; k < no; ++k) {
            int kk = oo[k];
            x += gi(g, N, i, a, kk, kk);
        }
        x *= parity_sign(X & between_mask(i, a));
        unsigned long long flip = (1ull << i) | (1ull << a);
        oa = alpha ? (A ^ flip) : A;
        ob = alpha ? B : (B ^ flip);
        return x;
    }
    if (e < P.seg[4]) {                       // same-spin doubles
        bool alpha = e < P.seg[3];
        long long idx = e - (alpha ? P.seg[2] : P.seg[3]);
        int cv = alpha ? P.cva2 : P.cvb2;
        int op = (int)(idx / cv), vp = (int)(idx - (long long)op * cv);
        unsigned short po = __ldg((alpha ? P.pair_oa : P.pair_ob) + op);
        unsigned short pv = __ldg((alpha ? P.pair_va : P.pair_vb) + vp);
        const unsigned char *os = alpha ? L.occA : L.occB;
        const unsigned char *vs = alpha ? L.virA : L.virB;
        int i = os[po & 0xff], j = os[po >> 8], a = vs[pv & 0xff], b = vs[pv >> 8];
        unsigned long long X = alpha ? A : B;
        double s1 = parity_sign(X & between_mask(i, a));
        unsigned long long X1 = X ^ (1ull << i) ^ (1ull << a);
        double s2 = parity_sign(X1 & between_mask(j, b));
        unsigned long long X2 = X1 ^ (1ull << j) ^ (1ull << b);
        double x = s1 * s2 * (gi(g, N, i, a, j, b) - gi(g, N, i, b, j, a));
        oa = alpha ? X2 : A;
        ob = alpha ? B : X2;
        return x;
    }
    // opposite-spin doubles
    long long idx = e - P.seg[4];
    long long nsb = (long long)P.nb * P.vb;
    int sa = (int)(idx / nsb);
    int sb = (int)(idx - (long long)sa * nsb);
    int oa_i = sa / P.va, va_i = sa - oa_i * P.va;
    int ob_i = sb / P.vb, vb_i = sb - ob_i * P.vb;
    int i = L.occA[oa_i], a = L.virA[va_i], j = L.occB[ob_i], b = L.virB[vb_i];
    double s = parity_sign(A & between_mask(i, a)) * parity_sign(B & between_mask(j, b));
    double x = s * gi(g, N, i, a, j, b);
    oa = A ^ (1ull << i) ^ (1ull << a);
    ob = B ^ (1ull << j) ^ (1ull << b);
    return x;
}

// Diagonal element: sum_p h_pp + sum_{p<q same spin} (J_pq - K_pq) + sum_{p alpha, q beta} J_pq,
// evaluated by one warp in a fixed order (lane-strided, then a butterfly sum).
__device__ __forceinline__ double diag_warp(const Problem &P, const ColLists &L) {
    const int lane = threadIdx.x & 31;
    const int N = P.N;
    double x = 0.0;
    for (int t = lane; t < P.na; t += 32) x += __ldg(P.h + L.occA[t] * (N + 1));
    for (int t = lane; t < P.nb; t += 32) x += __ldg(P.h + L.occB[t] * (N + 1));
    for (int t = lane; t < P.ca2; t += 32) {
        unsigned short pp = __ldg(P.pair_oa + t);
        int p = L.occA[pp & 0xff], q = L.occA[pp >> 8];
        x += __ldg(P.J + p * N + q) - __ldg(P.K + p * N + q);
    }
    for (int t = lane; t < P.cb2; t += 32) {
        unsigned short pp = __ldg(P.pair_ob + t);
        int p = L.occB[pp & 0xff], q = L.occB[pp >> 8];
        x += __ldg(P.J + p * N + q) - __ldg(P.K + p * N + q);
    }
    for (int t = lane; t < P.na * P.nb; t += 32) {
        int p = L.occA[t / P.nb], q = L.occB[t % P.nb];
        x += __ldg(P.J + p * N + q);
    }
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// ---------------------------------------------------------------------------
// Step size (appendix "Determining Step Size"): argmin of the quartic
// eta^4 + v3 eta^3 + v2 eta^2 + v1 eta.  Cardano's method on the cubic
// derivative gives the root(s) in single precision; each is refined by FP64
// Newton iterations on the cubic (the reciprocal of the derivative is taken
// in single precision, which keeps the iteration convergent and avoids an
// FP64 division).  With three real roots the outer two are refined and the
// one with the smaller quartic value is kept: that is the root farther from
// the middle one, the choice the appendix prescribes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double newton_cubic(double x, double v1, double v2, double v3) {
    for (int it = 0; it < 8; ++it) {
        double f = fma(fma(fma(4.0, x, 3.0 * v3), x, 2.0 * v2), x, v1);
        double fp = fma(fma(12.0, x, 6.0 * v3), x, 2.0 * v2);
        float fpf = (float)fp;
        if (fpf == 0.0f || !isfinite(fpf)) break;
        double step = f * (double)__frcp_rn(fpf);
        x -= step;
        if (fabs(step) <= 1e-15 * fabs(x)) break;
    }
    return x;
}

__device__ __forceinline__ double line_search(double v1, double v2, double v3) {
    const float b = 3.0f * (float)v3, c = 2.0f * (float)v2, d = (float)v1;
    const float sh = b * (1.0f / 12.0f);
    const float p = (12.0f * c - b * b) * (1.0f / 48.0f);
    const float q = (2.0f * b * b * b - 36.0f * b * c + 432.0f * d) * (1.0f / 1728.0f);
    const float hq = 0.5f * q, tp = p * (1.0f / 3.0f);
    const float del = hq * hq + tp * tp * tp;
    if (!(del < 0.0f) || !(p < 0.0f)) {
        float sd = sqrtf(fmaxf(del, 0.0f));
        float x = cbrtf(-hq + sd) + cbrtf(-hq - sd);
        return newton_cubic((double)(x - sh), v1, v2, v3);
    }
    float m = 2.0f * sqrtf(-tp);
    float arg = (3.0f * q / (2.0f * p)) * sqrtf(-3.0f / p);
    arg = fminf(1.0f, fmaxf(-1.0f, arg));
    float th = acosf(arg) * (1.0f / 3.0f);
    float xhi = m * cosf(th) - sh;                               // largest root
    float xlo = m * cosf(th - 4.18879020478639098f) - sh;        // smallest root (th - 4 pi / 3)
    double r1 = newton_cubic((double)xlo, v1, v2, v3);
    double r3 = newton_cubic((double)xhi, v1, v2, v3);
    double h1 = (((r1 + v3) * r1 + v2) * r1 + v1) * r1;
    double h3 = (((r3 + v3) * r3 + v2) * r3 + v1) * r3;
    return (h3 < h1) ? r3 : r1;
}

}  // namespace cdfci
