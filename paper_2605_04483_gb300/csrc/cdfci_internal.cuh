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
// Bit 63 of the beta word of a stored key marks "already a candidate" during a
// multicoordinate iteration (N <= 63 leaves it free); key comparisons ignore it.
constexpr unsigned long long kMarkB = 1ull << 63;
constexpr unsigned long long kKeyMaskB = ~kMarkB;
constexpr int kMaxPairs = 63 * 62 / 2;     // C(63, 2)
constexpr int kStatusOk = 0;

// error codes mirror include/cdfci.h
constexpr int kErrArg = -1, kErrNonfinite = -2, kErrTableFull = -3, kErrTimeout = -4,
              kErrNotNegative = -9, kErrInternal = -10;

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
// Dekker's shorter addition (relative error about 2^-104 instead of 2^-106):
// TwoSum of the leading parts, the trailing parts folded in once.
__host__ __device__ __forceinline__ dd dd_add_fast(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    return dd_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
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
// Per-handle device state between launches of the m = 1 cluster loop.
// ---------------------------------------------------------------------------
struct CdRecord {                  // written at the end of a launch, read at the start of the next
    unsigned long long a, b;       // coordinate i processed by launch l
    long long slot;
    double c_new;                  // c_i after the update
    double Hii;                    // H_ii
    double eta;                    // step of launch l
    dd mu, alpha;                  // c.c and c.Hc after the update (double-double)
    double mu_g;                   // the mu used in the gradients of the last column
    double dx, energy;
    long long iterations, nnz_c, n_slots, elements, applied, dropped, inserted, last_column;
    unsigned long long fa, fb;     // forced coordinate of the next step (a start vector's entry) ...
    double feta;                   // ... and its step (its c value)
    int forced;                    // 1: the next step takes (fa, fb) with eta = feta instead of the argmax
    int have_prev;                 // 1: (a, b, slot) was processed and the partials of its column are pending
    int done;                      // 1: dx < threshold; later launches only forward the state
};

struct __align__(16) CdPartial {   // per CTA: its share of the last processed column
    double gather;                 // sum_j H_ji c_j over this CTA's elements (for the recalculation of b_i)
    unsigned long long gbits;      // |4 b_j + 4 mu c_j| bits of this CTA's best candidate
    unsigned long long ka, kb;     // its key
    long long slot;                // its slot
    double bj, cj;                 // its b and c after the update
    int elements, applied, dropped, inserted;
    int err;                       // nonzero: this CTA hit an error (the status word holds the code)
};

// Control word and host-visible snapshot (one per handle).
struct IterState {
    int status;                    // first error code (sticky)
    int last_parity;               // parity of the most recent launch (its record is the current one)
    dd scale;                      // s: c_true = s * c_stored (1 for m = 1)
    // snapshot written by the finalisation kernel after each batch of launches
    long long iterations, nnz_c, n_slots, last_column, elements, applied, dropped, inserted;
    dd mu, alpha;
    double dx, energy, last_eta;
    unsigned long long last_a, last_b;
    long long eig_iters;           // m > 1: cumulative reduced-eigensolver iterations
    int done;
};

// Multicoordinate (m > 1) iteration state, one per handle.
struct McSel {                     // a chosen coordinate
    long long slot;
    unsigned long long gkey;       // |b + mu c| bits (the choice key)
    unsigned long long A, B;       // its determinant
};
struct McState {
    dd mu, alpha, scale;           // c.c, c.Hc (true units), global scale s (stored = true / s)
    double dx, energy, last_gamma;
    long long iterations, nnz_c, n_slots, elements, applied, dropped, inserted, last_column;
    unsigned long long cnt[4];     // counters of the running scatter
    unsigned long long sel_prefix; // radix selection: digits fixed so far
    int n_cand, m_sel, degenerate, done, done_pending;
    int sel_need, sel_level, sel_nbin, sel_resolved;
    int n_above, n_inbin;
    int eig_iters;                 // LOBPCG iterations of the last reduced problem
    long long eig_iters_total;
    // from the reduced solve to the update of mu and alpha that runs beside the scatter
    dd pend_scale;                 // s gamma
    double pend_gamma;
    int pend_it, pend_deg;
    // the finalisation's last-block counter and nonzero diagonals (zero between iterations)
    unsigned int fin_blocks;
    int fin_nd;
};

// xCDFCI (Algorithm 3, k1 = K + 1 states) iteration state, one per handle.
// Rows of C and B live beside the table: rows[slot * 2 k1 + a] = C_{slot,a},
// rows[slot * 2 k1 + k1 + a] = B_{slot,a}.
constexpr int kXMax = 8;
struct XState {
    dd S[kXMax * kXMax], M[kXMax * kXMax];   // C^T C, C^T H C (double-double)
    double g[kXMax];               // G_i of the chosen row (4 B_i + 4 C_i S)
    double wv[kXMax];              // scatter weights eta g
    double thr;                    // |H_ji| >= thr passes the compression rule: tau / max_a |eta g_a|
    double eta, dx, Hii;
    double E[kXMax];               // energies of the pencil (M, S), ascending (on request)
    long long slot;                // chosen row
    unsigned long long A, B;
    long long iterations, nnz_c, n_slots, elements, applied, dropped, inserted, last_column;
    unsigned long long cnt[4];     // counters of the running column
    int n_cand, k1, done;
};

// Everything a kernel needs about the problem and the table.
struct Problem {
    int N, na, nb, va, vb;
    int ca2, cb2, cva2, cvb2;      // C(na,2), C(nb,2), C(va,2), C(vb,2)
    long long seg[6];              // flat column segments: 0 diag | sa | sb | daa | dbb | dab | end=seg[5]
    long long nh;                  // enumeration length (= seg[5])
    int doubles_vanish;            // all (pq|rs) with p != q and r != s are zero (e.g. Hubbard)
    const double *h, *g, *J, *K;
    const double *W3, *V3;         // single-excitation terms, (i N + a) N + k: (ia|kk) - (ik|ka) and (ia|kk)
    const unsigned short *pair_oa, *pair_ob, *pair_va, *pair_vb;   // (i | j << 8), i < j
    Slot *table;
    unsigned long long mask;       // capacity - 1
    long long capacity;
    long long max_entries;         // floor(max_load * capacity)
    int max_probe;
    double tau;
    double theta, dx_threshold;
    unsigned long long mg_va, mg_vb, mg_nsb, mg_cva2, mg_cvb2;   // fdiv multipliers
    unsigned int *cnz;             // m > 1: filter of determinants whose c may be nonzero (NULL: none)
    unsigned long long cnz_mask;   // its bit count - 1
    unsigned int *mark;            // m > 1: candidate marks, one bit per slot (NULL: bit 63 of the slot's B)
    long long cap_cand;            // m > 1: entries of the candidate list
    // k-space Hubbard handles (cdfci_create_hubbard_k), else NULL: the index of the momentum
    // k_q - k_p (ksub[p N + q]) and of k_x + k_y (kadd[x N + y]); index 0 is k = 0
    const unsigned char *ksub, *kadd;
};

// k-space handles: an opposite-spin double with momentum transfers dA (alpha) and dB
// (beta) conserves momentum iff dA + dB = 0; the others are zero without an integral load.
__device__ __forceinline__ bool k_conserved(const Problem &P, int dA, int dB) {
    return !P.kadd || __ldg(P.kadd + dA * P.N + dB) == 0;
}

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
// x times (-1)^popcount(m), as a flip of the sign bit (exact, no FP64 operation)
__device__ __forceinline__ double apply_parity(double x, unsigned long long m) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)(__popcll(m) & 1) << 63));
}
// SplitMix64 output finalizer (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
// Slot hash of a determinant: the xor of independent hashes of its alpha and
// beta strings (two-character tabulation-style combination), so that the
// hash of an excitation can be assembled from per-column tables.
__host__ __device__ __forceinline__ unsigned long long hash_alpha(unsigned long long a) {
    return mix64(a ^ 0x9e3779b97f4a7c15ull);
}
__host__ __device__ __forceinline__ unsigned long long hash_beta(unsigned long long b) {
    return mix64(b ^ 0xd1b54a32d192ed03ull);
}
__host__ __device__ __forceinline__ unsigned long long key_hash(unsigned long long a, unsigned long long b) {
    return hash_alpha(a) ^ hash_beta(b);
}

// Filter of determinants whose c may be nonzero: one bit per bucket of the
// high half of the key's hash (the table's slot comes from the low bits).  A
// clear bit proves c = 0; bits are set wherever a c becomes nonzero and never
// cleared, so a set bit only means "look it up".
__device__ __forceinline__ void cnz_set(const Problem &P, unsigned long long a, unsigned long long b) {
    if (!P.cnz) return;
    const unsigned long long i = (key_hash(a, b) >> 32) & P.cnz_mask;
    atomicOr(P.cnz + (i >> 5), 1u << (unsigned)(i & 31));
}
__device__ __forceinline__ bool cnz_maybe(const Problem &P, unsigned long long h) {
    if (!P.cnz) return true;
    const unsigned long long i = (h >> 32) & P.cnz_mask;
    return (__ldg(P.cnz + (i >> 5)) >> (unsigned)(i & 31)) & 1u;
}

// Candidate mark of slot s in the m > 1 bitmap: set (returns true if this call set it), test, clear.
__device__ __forceinline__ bool mark_set(const Problem &P, long long s) {
    const unsigned bit = 1u << (unsigned)(s & 31);
    return !(atomicOr(P.mark + (s >> 5), bit) & bit);
}
__device__ __forceinline__ bool mark_test(const Problem &P, long long s) {
    return (P.mark[s >> 5] >> (unsigned)(s & 31)) & 1u;
}
__device__ __forceinline__ void mark_clear(const Problem &P, long long s) {
    atomicAnd(P.mark + (s >> 5), ~(1u << (unsigned)(s & 31)));
}

// floor(n / d) for n < 2^24, d < 2^16 with M = floor(2^40 / d) + 1 (the
// rounding error n (M - 2^40/d) / 2^40 < 1/d cannot reach the next integer).
__host__ __device__ __forceinline__ unsigned fdiv(unsigned n, unsigned long long M) {
    return (unsigned)(((unsigned long long)n * M) >> 40);
}
__host__ __forceinline__ unsigned long long fdiv_magic(unsigned d) { return d ? (1ull << 40) / d + 1 : 0; }

// +0.0 or -0.0, tested on the bit pattern (keeps the test off the FP64 pipe)
__device__ __forceinline__ bool is_zero(double x) { return ((unsigned long long)__double_as_longlong(x) << 1) == 0ull; }
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

// Programmatic dependent launch (sm_90+): wait for the preceding grid's
// completion and memory, and let the next grid start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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
        if (ka == a && (kb & kKeyMaskB) == b) return (long long)pos;
        if (ka == 0ull && kb == 0ull) {
            if (!insert) return -1;
            unsigned long long oa, ob;
            cas128(&s->a, 0ull, 0ull, a, b, oa, ob);
            if (oa == 0ull && ob == 0ull) { *inserted = true; return (long long)pos; }
            // lost to an insert of the same key (which may already carry the candidate mark)
            if (oa == a && (ob & kKeyMaskB) == b) return (long long)pos;
        }
        pos = (pos + 1) & P.mask;
    }
    set_status(st, kErrTableFull);
    return -2;
}

// The grid-wide m = 1 loop (all CTAs co-resident: cooperative launch) hands
// every round's CTA partials over through an exchange buffer whose words carry
// the number of the round that wrote them, so a reader polls the data itself
// instead of a barrier counter.  `round` counts the rounds published by earlier
// launches (zero-initialised, never reset).
struct GridRound {
    unsigned long long round;
};
// 64-bit words per CTA partial in the exchange buffer: word k holds 32-bit
// half k of the CdPartial in its low half and the round (mod 2^32) in its high
// half, so every word validates itself (a 64-bit access is single-copy atomic;
// a vector access is not as a whole).  Two buffers of G partials alternate.
constexpr int kXchgWords = 20;
static_assert(sizeof(CdPartial) == 4 * kXchgWords, "CdPartial is exchanged as 32-bit halves");

// One problem of a batch of independent m = 1 solvers stepped in one launch.
struct CdInstance {
    Problem P;
    IterState *st;
    CdRecord *rec;
    CdPartial *part;
};

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

// A decoded column element: which excitation of the column determinant.
struct ElemIdx {
    int kind;                          // 0 single alpha, 1 single beta, 2 double aa, 3 double bb, 4 double ab
    int i, a, j, b;                    // orbitals (j, b unused for singles)
    unsigned long long sgn;            // bits whose parity gives the sign (two masks folded by xor)
    int gidx;                          // for kind 4: index of (ia|jb) in g, or -1
};

// Integer part of column element e in [1, nh): the excitation and the key D'.
// Signs: the bits of the same-spin string strictly between the two orbitals
// of each elementary excitation, applied in the order i->a then j->b.
__device__ __forceinline__ void decode_element(const Problem &P, const ColLists &L, unsigned long long A,
                                               unsigned long long B, long long e, unsigned long long &oa,
                                               unsigned long long &ob, ElemIdx &x) {
    if (e < P.seg[2]) {                       // singles
        const bool alpha = e < P.seg[1];
        const unsigned idx = (unsigned)(e - (alpha ? P.seg[0] : P.seg[1]));
        const unsigned v = (unsigned)(alpha ? P.va : P.vb);
        const int o = (int)fdiv(idx, alpha ? P.mg_va : P.mg_vb), w = (int)(idx - (unsigned)o * v);
        const int i = alpha ? L.occA[o] : L.occB[o];
        const int a = alpha ? L.virA[w] : L.virB[w];
        const unsigned long long X = alpha ? A : B;
        const unsigned long long flip = (1ull << i) | (1ull << a);
        x.kind = alpha ? 0 : 1;
        x.i = i; x.a = a; x.j = 0; x.b = 0;
        x.sgn = X & between_mask(i, a);
        x.gidx = -1;
        oa = alpha ? (A ^ flip) : A;
        ob = alpha ? B : (B ^ flip);
        return;
    }
    if (e < P.seg[4]) {                       // same-spin doubles
        const bool alpha = e < P.seg[3];
        const unsigned idx = (unsigned)(e - (alpha ? P.seg[2] : P.seg[3]));
        const unsigned cv = (unsigned)(alpha ? P.cva2 : P.cvb2);
        const int op = (int)fdiv(idx, alpha ? P.mg_cva2 : P.mg_cvb2), vp = (int)(idx - (unsigned)op * cv);
        const unsigned short po = __ldg((alpha ? P.pair_oa : P.pair_ob) + op);
        const unsigned short pv = __ldg((alpha ? P.pair_va : P.pair_vb) + vp);
        const unsigned char *os = alpha ? L.occA : L.occB;
        const unsigned char *vs = alpha ? L.virA : L.virB;
        const int i = os[po & 0xff], j = os[po >> 8], a = vs[pv & 0xff], b = vs[pv >> 8];
        const unsigned long long X = alpha ? A : B;
        const unsigned long long m1 = X & between_mask(i, a);
        const unsigned long long X1 = X ^ (1ull << i) ^ (1ull << a);
        const unsigned long long m2 = X1 & between_mask(j, b);
        const unsigned long long X2 = X1 ^ (1ull << j) ^ (1ull << b);
        x.kind = alpha ? 2 : 3;
        x.i = i; x.a = a; x.j = j; x.b = b;
        x.sgn = m1 ^ m2;
        x.gidx = -1;                      // popcount parity of m1 ^ m2 = parity(m1) xor parity(m2)
        oa = alpha ? X2 : A;
        ob = alpha ? B : X2;
        return;
    }
    const unsigned idx = (unsigned)(e - P.seg[4]);   // opposite-spin doubles
    const unsigned nsb = (unsigned)(P.nb * P.vb);
    const unsigned sa = fdiv(idx, P.mg_nsb);
    const unsigned sb = idx - sa * nsb;
    const int oa_i = (int)fdiv(sa, P.mg_va), va_i = (int)(sa - (unsigned)oa_i * (unsigned)P.va);
    const int ob_i = (int)fdiv(sb, P.mg_vb), vb_i = (int)(sb - (unsigned)ob_i * (unsigned)P.vb);
    const int i = L.occA[oa_i], a = L.virA[va_i], j = L.occB[ob_i], b = L.virB[vb_i];
    x.kind = 4;
    x.i = i; x.a = a; x.j = j; x.b = b;
    x.sgn = (A & between_mask(i, a)) ^ (B & between_mask(j, b));
    x.gidx = -1;
    oa = A ^ (1ull << i) ^ (1ull << a);
    ob = B ^ (1ull << j) ^ (1ull << b);
}

// Value part (Eq. entry): singles h_ia + sum over the occupied spin-orbitals k
// of the column determinant, taken in spin-orbital order (alpha ascending, then
// beta ascending), of (ia|kk) - (ik|ka) for k of the single's spin and (ia|kk)
// for the other spin, one running sum in exactly that order (so the value does
// not depend on the kernel or on which of the two determinants is the column);
// same-spin doubles (ia|jb) - (ib|ja); opposite-spin doubles (ia|jb); all times
// the sign.
__device__ __forceinline__ double element_value(const Problem &P, const ColLists &L, const ElemIdx &x) {
    const int N = P.N;
    const double *g = P.g;
    double v;
    if (x.kind <= 1) {
        const bool alpha = x.kind == 0;
        const int i = x.i, a = x.a;
        v = __ldg(P.h + i * N + a);
        for (int k = 0; k < P.na; ++k) {
            const int kk = L.occA[k];
            const double t = gi(g, N, i, a, kk, kk);
            v += alpha ? t - gi(g, N, i, kk, kk, a) : t;
        }
        for (int k = 0; k < P.nb; ++k) {
            const int kk = L.occB[k];
            const double t = gi(g, N, i, a, kk, kk);
            v += alpha ? t : t - gi(g, N, i, kk, kk, a);
        }
    } else if (x.kind <= 3) {
        v = gi(g, N, x.i, x.a, x.j, x.b) - gi(g, N, x.i, x.b, x.j, x.a);
    } else {
        v = x.gidx >= 0 ? __ldg(g + x.gidx) : gi(g, N, x.i, x.a, x.j, x.b);
    }
    return apply_parity(v, x.sgn);
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// One single excitation of the column determinant (per-iteration table): the
// changed string, its hash, the offset of its orbital pair in g, the sign, the
// orbitals and, for k-space handles, the momentum transfer k_a - k_i
// (info = sign | i << 8 | a << 16 | transfer << 24).
struct SingleEnt {
    unsigned long long key, h;
    int goff;                          // alpha table: (i N + a) N^2;  beta table: j N + b
    int info;
};

__device__ __forceinline__ int j_b_off(int N, int j, int b) { return j * N + b; }

__device__ __forceinline__ void build_singles(const Problem &P, const ColLists &L, unsigned long long iA,
                                              unsigned long long iB, SingleEnt *tabA, SingleEnt *tabB, int t0, int nt) {
    const int na_va = P.na * P.va, nb_vb = P.nb * P.vb, N = P.N;
    for (int s = t0; s < na_va + nb_vb; s += nt) {
        const bool alpha = s < na_va;
        const int sl = alpha ? s : s - na_va;
        const int o = (int)fdiv((unsigned)sl, alpha ? P.mg_va : P.mg_vb);
        const int w = sl - o * (alpha ? P.va : P.vb);
        const int i = alpha ? L.occA[o] : L.occB[o];
        const int a = alpha ? L.virA[w] : L.virB[w];
        const unsigned long long X = alpha ? iA : iB;
        SingleEnt e;
        e.key = X ^ (1ull << i) ^ (1ull << a);
        e.h = alpha ? hash_alpha(e.key) : hash_beta(e.key);
        e.goff = alpha ? (i * N + a) * N * N : j_b_off(N, i, a);
        e.info = (__popcll(X & between_mask(i, a)) & 1) | (i << 8) | (a << 16) |
                 (P.ksub ? (int)__ldg(P.ksub + i * N + a) << 24 : 0);
        (alpha ? tabA : tabB)[sl] = e;
    }
}

// One element of the column of {A, B}: flat index e in [1, nh).  Returns the
// value H_{D',D} (0.0 when the Slater-Condon element vanishes) and the key D'.
__device__ __forceinline__ double column_element(const Problem &P, const ColLists &L, unsigned long long A,
                                                 unsigned long long B, long long e, unsigned long long &oa,
                                                 unsigned long long &ob) {
    ElemIdx x;
    decode_element(P, L, A, B, e, oa, ob, x);
    return element_value(P, L, x);
}

// Diagonal element: sum_p h_pp + sum_{p<q same spin} (J_pq - K_pq) + sum_{p alpha, q beta} J_pq,
// evaluated by one warp in a fixed order (lane-strided over all ordered pairs
// of occupied spin-orbitals, then a shuffle-down tree; every lane returns the
// same value).  An ordered same-spin pair contributes (J - K) / 2, an ordered
// opposite-spin pair J / 2, so each unordered pair is counted once.
// J and K may be global or shared memory (the loop kernels stage them in
// shared memory).  A lane's pair terms t = lane + 32 r go to four partial sums
// (r mod 4) whose loads are independent, combined pairwise.
__device__ __forceinline__ double diag_warp(const Problem &P, const ColLists &L, const double *J, const double *K) {
    const int lane = threadIdx.x & 31;
    const int N = P.N, n = P.na + P.nb, n2 = n * n;
    double x = 0.0;
    for (int t = lane; t < n; t += 32) {
        const int p = t < P.na ? L.occA[t] : L.occB[t - P.na];
        x += __ldg(P.h + p * (N + 1));
    }
    double y4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t0 = lane; t0 < n2; t0 += 128) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int t = t0 + 32 * r;
            if (t >= n2) continue;
            const int u = t / n, w = t - u * n;
            if (u == w) continue;
            const bool ua = u < P.na, wa = w < P.na;
            const int p = ua ? L.occA[u] : L.occB[u - P.na];
            const int q = wa ? L.occA[w] : L.occB[w - P.na];
            const double jv = J[p * N + q];
            y4[r] += (ua == wa) ? (jv - K[p * N + q]) : jv;
        }
    }
    x = fma(0.5, (y4[0] + y4[1]) + (y4[2] + y4[3]), x);
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    return __shfl_sync(0xffffffffu, x, 0);
}
__device__ __forceinline__ double diag_warp(const Problem &P, const ColLists &L) {
    return diag_warp(P, L, P.J, P.K);
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
// Reciprocal of d to about 1e-14 relative: single-precision estimate plus one
// Newton-Raphson correction in FP64.
__device__ __forceinline__ double recip(double d) {
    const double r = (double)__frcp_rn((float)d);
    return fma(r, fma(-d, r, 1.0), r);
}

// One Halley step (cubic convergence) on 4x^3 + 3 v3 x^2 + 2 v2 x + v1 = 0.
__device__ __forceinline__ double halley_cubic(double x, double v1, double v2, double v3) {
    const double f = fma(fma(fma(4.0, x, 3.0 * v3), x, 2.0 * v2), x, v1);
    const double f1 = fma(fma(12.0, x, 6.0 * v3), x, 2.0 * v2);
    const double f2 = fma(24.0, x, 6.0 * v3);
    const double den = fma(2.0 * f1, f1, -f * f2);
    if (!(den != 0.0) || !isfinite(den)) return x;
    return x - 2.0 * f * f1 * recip(den);
}

// Two single-precision Newton steps on the cubic in eta itself (so a root
// near 0 keeps its relative accuracy).
__device__ __forceinline__ float newton_f32(float x, float v1, float v2, float v3) {
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const float f = fmaf(fmaf(fmaf(4.0f, x, 3.0f * v3), x, 2.0f * v2), x, v1);
        const float f1 = fmaf(fmaf(12.0f, x, 6.0f * v3), x, 2.0f * v2);
        if (f1 != 0.0f) x -= f * __frcp_rn(f1);
    }
    return x;
}

// Cube root to about 1e-6 relative from the special-function unit's base-2
// logarithm and exponential (0 for 0); it only seeds the Newton steps below.
__device__ __forceinline__ float cbrt_seed(float x) {
    return copysignf(exp2f(__log2f(fabsf(x)) * (1.0f / 3.0f)), x);
}

// Step size (appendix "Determining Step Size"): the global minimiser of
// eta^4 + v3 eta^3 + v2 eta^2 + v1 eta.  Cardano's method on the cubic
// derivative, with the depressed cubic in single precision; the chosen root is
// polished by two single-precision Newton steps in eta and one FP64 Halley
// step.  With three real roots x1 < x2 < x3 the minimum at x3 is lower exactly
// when x3 - x2 > x2 - x1 (the quartic's difference between them is
// -(x3 - x1)^3 ((x3 - x2) - (x2 - x1)) / 3), so the root farther from the
// middle one wins, x1 on a tie.  A tie is a difference of the two distances
// below 1e-9 of their sum (e.g. a coordinate that is the only nonzero one,
// whose quartic is symmetric about -c_i): decided in single precision when
// the distances differ by more than 1e-4 of their sum, else on the FP64
// roots through the quartic's values and that identity.
__device__ __forceinline__ double line_search(double v1, double v2, double v3) {
    const float f1 = (float)v1, f2 = (float)v2, f3 = (float)v3;
    const float b = 3.0f * f3, c = 2.0f * f2, d = f1;
    const float sh = b * (1.0f / 12.0f);
    const float p = (12.0f * c - b * b) * (1.0f / 48.0f);
    const float q = (2.0f * b * b * b - 36.0f * b * c + 432.0f * d) * (1.0f / 1728.0f);
    const float hq = 0.5f * q, tp = p * (1.0f / 3.0f);
    const float del = hq * hq + tp * tp * tp;
    if (!(del < 0.0f) || !(p < 0.0f)) {
        const float sd = sqrtf(fmaxf(del, 0.0f));
        const float x = cbrt_seed(-hq + sd) + cbrt_seed(-hq - sd) - sh;
        return halley_cubic((double)newton_f32(x, f1, f2, f3), v1, v2, v3);
    }
    const float m = 2.0f * sqrtf(-tp);
    float arg = (3.0f * q / (2.0f * p)) * sqrtf(-3.0f / p);
    arg = fminf(1.0f, fmaxf(-1.0f, arg));
    const float th = acosf(arg) * (1.0f / 3.0f);
    const float x3 = m * cosf(th);                            // depressed roots x1 <= x2 <= x3
    const float x2 = m * cosf(th - 2.09439510239319549f);
    const float x1 = m * cosf(th - 4.18879020478639098f);
    const float d1 = x2 - x1, d3 = x3 - x2;
    if (d3 - d1 > 1e-4f * (d1 + d3)) return halley_cubic((double)newton_f32(x3 - sh, f1, f2, f3), v1, v2, v3);
    if (d1 - d3 > 1e-4f * (d1 + d3)) return halley_cubic((double)newton_f32(x1 - sh, f1, f2, f3), v1, v2, v3);
    const double r1 = halley_cubic((double)newton_f32(x1 - sh, f1, f2, f3), v1, v2, v3);
    const double r3 = halley_cubic((double)newton_f32(x3 - sh, f1, f2, f3), v1, v2, v3);
    const double h1 = (((r1 + v3) * r1 + v2) * r1 + v1) * r1;
    const double h3 = (((r3 + v3) * r3 + v2) * r3 + v1) * r3;
    const double w = r3 - r1;
    // x3 iff (d3 - d1) > 1e-9 (d1 + d3), i.e. h1 - h3 > 1e-9 / 3 (x3 - x1)^4
    return (h1 - h3 > (1e-9 / 3.0) * (w * w) * (w * w)) ? r3 : r1;
}

}  // namespace cdfci
