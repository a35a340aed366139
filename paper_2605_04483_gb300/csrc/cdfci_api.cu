// Host side of the libcdfci C-ABI (include/cdfci.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <new>
#include <string>
#include <map>
#include <vector>

#include "../../include/cdfci.h"
#include "cdfci_internal.cuh"
#include "cdfci_kernels.h"

using namespace cdfci;

// The grid-wide m = 1 loop exchanges a CdPartial as 32-bit halves in this field
// order (the loop kernel's xchg_unpack reads them back by offset).
static_assert(offsetof(CdPartial, gather) == 0 && offsetof(CdPartial, gbits) == 8 && offsetof(CdPartial, ka) == 16 &&
                  offsetof(CdPartial, kb) == 24 && offsetof(CdPartial, slot) == 32 && offsetof(CdPartial, bj) == 40 &&
                  offsetof(CdPartial, cj) == 48 && offsetof(CdPartial, elements) == 56 &&
                  offsetof(CdPartial, applied) == 60 && offsetof(CdPartial, dropped) == 64 &&
                  offsetof(CdPartial, inserted) == 68 && offsetof(CdPartial, err) == 72,
              "CdPartial layout of the partial exchange");

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(CDFCI_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaMemcpyKind kind_to_device(const void *src) {
    return is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}

long long binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

std::vector<unsigned short> pair_table(int n) {
    std::vector<unsigned short> t;
    for (int j = 1; j < n; ++j)
        for (int i = 0; i < j; ++i) t.push_back((unsigned short)(i | (j << 8)));
    return t;
}

}  // namespace

void cdfci::set_last_error_message(const char *msg) { g_last_error = msg; }

struct cdfci_ctx {
    cdfci_params prm;                            // as given (log2_capacity resolved from max_memory)
    int N, na, nb;
    Problem P;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // device buffers
    double *d_h = nullptr, *d_g = nullptr, *d_J = nullptr, *d_K = nullptr, *d_W3 = nullptr, *d_V3 = nullptr;
    unsigned short *d_pairs = nullptr;
    unsigned char *d_ktab = nullptr;   // k-space handles: ksub then kadd (N x N each)
    Slot *d_table = nullptr;
    IterState *d_st = nullptr;
    CdRecord *d_rec = nullptr;                   // state between launches of the cluster loop
    CdPartial *d_part = nullptr;                 // one partial per CTA of the cluster (two sets in grid mode)
    GridRound *d_bar = nullptr;                  // grid mode: rounds of the partial exchange so far
    bool gridmode = false;                       // m = 1 over more CTAs than a cluster holds
    int *d_flags = nullptr;                      // [0] status, [1] has_doubles
    unsigned long long *d_counter = nullptr;     // scratch counter for compaction kernels
    unsigned long long *d_colkeys = nullptr;     // get_column staging (2 * nh)
    double *d_colvals = nullptr;
    IterState *h_st = nullptr;                   // pinned copy of the state
    int grid = 1;                                // CTAs of the cluster
    long long chunk = 1 << 16;                   // iterations per launch
    // multicoordinate (m > 1) iteration
    bool block = false;
    McBuffers mb;
    void *mb_alloc[32] = {};
    int mb_nalloc = 0;
    int mchunk = 8;                              // iterations per captured graph
    cudaGraphExec_t mgraph = nullptr;
    int tau_raises = 0;                          // z_threshold_search: tenfold raises so far
    // xCDFCI (num_states = K + 1 > 1)
    bool xcd = false;
    int k1 = 1;
    XBuffers xb{};
};

namespace {

void free_ctx(cdfci_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->mgraph) cudaGraphExecDestroy(c->mgraph);
    for (int i = 0; i < c->mb_nalloc; ++i) cudaFree(c->mb_alloc[i]);
    cudaFree(c->d_h); cudaFree(c->d_g); cudaFree(c->d_J); cudaFree(c->d_K); cudaFree(c->d_W3); cudaFree(c->d_V3);
    cudaFree(c->d_pairs); cudaFree(c->d_ktab); cudaFree(c->d_table); cudaFree(c->d_st); cudaFree(c->d_part); cudaFree(c->d_rec);
    cudaFree(c->d_bar);
    cudaFree(c->d_flags); cudaFree(c->d_counter); cudaFree(c->d_colkeys); cudaFree(c->d_colvals);
    if (c->h_st) cudaFreeHost(c->h_st);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int fill_stats(cdfci_ctx *c, cdfci_stats *s);
int exact_rq(cdfci_ctx *c, const Problem &P, double *E);

// z_threshold_search: the r-th tenfold raise of tau comes when the stored determinants pass
// 1 - 2^-(r+1) of max_entries (50 %, 75 %, 87.5 %, ...), so each raise leaves half of the
// remaining room; the first raise starts from at least 1e-6 |E| (the scale of H) or 1e-10.
// Reads the snapshot first; *changed tells whether tau moved.
int maybe_raise_tau(cdfci_ctx *c, bool *changed) {
    *changed = false;
    if (!c->prm.z_threshold_search) return CDFCI_OK;
    int rc = fill_stats(c, nullptr);
    if (rc) return rc;
    const double frac = 1.0 - std::ldexp(1.0, -(c->tau_raises + 1));
    if ((double)c->h_st->n_slots >= frac * (double)c->P.max_entries) {
        c->P.tau = std::max({10.0 * c->P.tau, 1e-6 * std::fabs(c->h_st->energy), 1e-10});
        c->tau_raises += 1;
        *changed = true;
    }
    return CDFCI_OK;
}

int run_iterations(cdfci_ctx *c, long long n) {
    const long long chunk = c->prm.z_threshold_search ? std::min<long long>(c->chunk, 1024) : c->chunk;
    while (n > 0) {
        bool changed = false;
        int rc = maybe_raise_tau(c, &changed);
        if (rc) return rc;
        long long k = std::min(n, chunk);
        if (c->gridmode)
            CK(launch_cd_loop_grid(c->P, c->d_st, c->d_rec, c->d_part,
                                   reinterpret_cast<unsigned long long *>(c->d_part + c->grid), c->d_bar, c->grid, k,
                                   c->stream));
        else
            CK(launch_cd_loop(c->P, c->d_st, c->d_rec, c->d_part, c->grid, k, c->stream));
        n -= k;
    }
    return CDFCI_OK;
}

int stats_from_snapshot(cdfci_ctx *c, cdfci_stats *s);

int fill_stats(cdfci_ctx *c, cdfci_stats *s) {
    if (c->xcd) CK(launch_x_energies(c->xb, c->stream));
    else if (!c->block) CK(launch_cd_finalize(c->P, c->d_st, c->d_rec, c->d_part, c->grid, c->stream));
    CK(cudaMemcpyAsync(c->h_st, c->d_st, sizeof(IterState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return stats_from_snapshot(c, s);
}

// the host snapshot c->h_st as cdfci_stats; the sticky device status as the return code
int stats_from_snapshot(cdfci_ctx *c, cdfci_stats *s) {
    const IterState &t = *c->h_st;
    if (s) {
        s->iterations = t.iterations;
        s->energy = t.energy;
        s->mu = t.mu.hi;
        s->alpha = t.alpha.hi;
        s->dx = t.dx;
        s->nnz_c = t.nnz_c;
        s->n_slots = t.n_slots;
        s->last_column = t.last_column;
        s->elements = t.elements;
        s->applied = t.applied;
        s->dropped = t.dropped;
        s->inserted = t.inserted;
        s->load = (double)t.n_slots / (double)c->P.capacity;
        s->status = t.status;
        s->converged = t.done;
        s->reduced_iterations = t.eig_iters;
        s->grid_blocks = (c->block || c->xcd) ? 0 : c->grid;
        s->grid_wide = c->gridmode ? 1 : 0;
        s->z_threshold = c->P.tau;
    }
    if (t.status != 0) {
        const char *what = t.status == CDFCI_ERR_TABLE_FULL ? "hash table full (raise log2_capacity or z_threshold)"
                           : t.status == CDFCI_ERR_NONFINITE ? "non-finite value in an update"
                           : t.status == CDFCI_ERR_TIMEOUT   ? "bounded device wait expired"
                           : t.status == CDFCI_ERR_INTERNAL  ? "device consistency check failed"
                                                             : "device error";
        return fail(t.status, "%s", what);
    }
    return CDFCI_OK;
}

template <typename T>
int mb_alloc(cdfci_ctx *c, T **p, size_t count) {
    if (cudaMalloc((void **)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return -1;
    c->mb_alloc[c->mb_nalloc++] = (void *)*p;
    return cudaMemsetAsync(*p, 0, std::max<size_t>(count, 1) * sizeof(T), c->stream) == cudaSuccess ? 0 : -1;
}

int setup_block(cdfci_ctx *c, int m) {
    McBuffers &b = c->mb;
    const Problem &P = c->P;
    const long long nh_eff = P.doubles_vanish ? P.seg[2] : P.seg[5];
    b.m = m;
    const long long cap_cand = (long long)m * nh_eff + m + 64;
    b.cap_cand = cap_cand;
    c->P.cap_cand = cap_cand;
    CK(mc_configure());
    b.geom = mc_geometry(P);
    // grids sized to the problem's work (a small problem leaves the rest of the GPU to the other
    // problems of a batch): the scatter's warps take about two items each, at most the resident
    // blocks; the candidate passes give every thread at least eight candidates, at most 4 blocks per SM
    const int resident = mc_scatter_grid(P);
    if (resident <= 0) return fail(CDFCI_ERR_CUDA, "occupancy query of the scatter failed");
    const long long items = (long long)m * b.geom.per_col;
    b.scatter_grid = (int)std::max<long long>(1, std::min<long long>(resident, (items + 15) / 16));
    b.cand_grid = (int)std::max<long long>(1, std::min<long long>(152 * 4, (cap_cand + 2047) / 2048));
    const size_t ns = (size_t)b.geom.nsA + (size_t)b.geom.nsB;
    b.st = c->d_st;
    const size_t n1 = (size_t)m + 1;
    b.ldr = mc_ldr(m);
    if (mb_alloc(c, &b.ms, 1) || mb_alloc(c, &b.cand, (size_t)cap_cand) || mb_alloc(c, &b.gkey, (size_t)cap_cand) ||
        mb_alloc(c, &b.hist, 4096 + 1) || mb_alloc(c, &b.sel, (size_t)m) || mb_alloc(c, &b.inbin, 4096) || mb_alloc(c, &b.ties, (size_t)cap_cand) ||
        mb_alloc(c, &b.cI, (size_t)m) || mb_alloc(c, &b.bI, (size_t)m) || mb_alloc(c, &b.Hdiag, (size_t)m) ||
        mb_alloc(c, &b.HIIc, (size_t)m) || mb_alloc(c, &b.Rh, n1 * (size_t)b.ldr) ||
        mb_alloc(c, &b.Rl, n1 * (size_t)b.ldr) ||
        mb_alloc(c, &b.w, (size_t)m) || mb_alloc(c, &b.thr, (size_t)m) || mb_alloc(c, &b.eta, (size_t)m) ||
        mb_alloc(c, &b.gathp, (size_t)m * (size_t)b.geom.per_col) || mb_alloc(c, &b.coltab, (size_t)m * ns) ||
        mb_alloc(c, &b.collists, (size_t)m) || mb_alloc(c, &b.work, 1) || mb_alloc(c, &b.rowf, 2 * (size_t)m))
        return fail(CDFCI_ERR_NOMEM, "allocation of the multicoordinate buffers failed");
    // c != 0 filter: one bit per table slot, between 2^16 and 2^25 bits (4 MB: it stays in L2 while the
    // scatter's random slot traffic streams through)
    const unsigned long long nbits =
        (unsigned long long)std::min<long long>(std::max<long long>(P.capacity, 1ll << 16), 1ll << 25);
    if (mb_alloc(c, &c->P.cnz, (size_t)(nbits / 32)))
        return fail(CDFCI_ERR_NOMEM, "allocation of the multicoordinate buffers failed");
    c->P.cnz_mask = nbits - 1;
    // candidate marks: one bit per slot
    if (mb_alloc(c, &c->P.mark, (size_t)((P.capacity + 31) / 32)))
        return fail(CDFCI_ERR_NOMEM, "allocation of the multicoordinate buffers failed");
    return CDFCI_OK;
}

// xCDFCI buffers and the start rows: the reference and the K determinants of
// its column with the lowest diagonal (ties: the smaller key).
int setup_xcd(cdfci_ctx *c, int k1, unsigned long long refA, unsigned long long refB) {
    XBuffers &b = c->xb;
    const Problem &P = c->P;
    cudaStream_t s = c->stream;
    const long long nh_eff = P.doubles_vanish ? P.seg[2] : P.seg[5];
    c->k1 = k1;
    b.nscatter = x_scatter_blocks();
    b.nselect = 152;
    b.cap_cand = (long long)k1 * (nh_eff + 1) + 64;
    if (mb_alloc(c, &b.xs, 1) || mb_alloc(c, &b.rows, (size_t)P.capacity * 2 * k1) ||
        mb_alloc(c, &b.cand, (size_t)b.cap_cand) || mb_alloc(c, &b.gathp, (size_t)b.nscatter * k1) ||
        mb_alloc(c, reinterpret_cast<unsigned char **>(&b.bbest), (size_t)b.nselect * x_block_bytes()) ||
        mb_alloc(c, &b.counter, 1))
        return fail(CDFCI_ERR_NOMEM, "device allocation of the xCDFCI buffers failed");
    b.st = c->d_st;
    XState x;
    memset(&x, 0, sizeof(x));
    x.k1 = k1;
    CK(cudaMemcpyAsync(b.xs, &x, sizeof(x), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(b.rows, 0, (size_t)P.capacity * 2 * k1 * sizeof(double), s));
    CK(cudaMemsetAsync(b.counter, 0, sizeof(unsigned int), s));
    // the reference column and its diagonals
    CK(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), s));
    CK(launch_column(P, refA, refB, c->d_colkeys, c->d_colvals, P.nh, c->d_counter, s));
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, c->d_counter, sizeof(n), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<unsigned long long> keys(2 * n);
    std::vector<double> diag(n);
    double *dd_ = nullptr;
    if (n > 0) {
        if (cudaMalloc(&dd_, n * sizeof(double)) != cudaSuccess) return fail(CDFCI_ERR_NOMEM, "device allocation failed");
        cudaError_t e = launch_x_diag_list(P, c->d_colkeys, (long long)n, dd_, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(keys.data(), c->d_colkeys, 2 * n * sizeof(unsigned long long),
                                                  cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(diag.data(), dd_, n * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(dd_);
        if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "start rows: %s", cudaGetErrorString(e));
    }
    struct Cand { double d; unsigned long long a, b; };
    std::vector<Cand> cs;
    for (unsigned long long k = 0; k < n; ++k)
        if (!(keys[2 * k] == refA && keys[2 * k + 1] == refB)) cs.push_back({diag[k], keys[2 * k], keys[2 * k + 1]});
    std::sort(cs.begin(), cs.end(), [](const Cand &x, const Cand &y) {
        if (x.d != y.d) return x.d < y.d;
        return x.b != y.b ? x.b < y.b : x.a < y.a;
    });
    if ((int)cs.size() < k1 - 1)
        return fail(CDFCI_ERR_ARG, "num_states = %d: the reference column has only %d other determinants", k1,
                    (int)cs.size());
    CK(launch_x_start(P, b, refA, refB, 0, s));
    for (int k = 1; k < k1; ++k) CK(launch_x_start(P, b, cs[k - 1].a, cs[k - 1].b, k, s));
    return CDFCI_OK;
}

int build_xcd_graph(cdfci_ctx *c) {
    cudaGraph_t got = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < c->mchunk && e == cudaSuccess; ++i) e = launch_x_iteration(c->P, c->xb, c->stream);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &got);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (got) cudaGraphDestroy(got);
        return fail(CDFCI_ERR_CUDA, "capture of the xCDFCI iteration failed");
    }
    e = cudaGraphInstantiate(&c->mgraph, got, 0);
    cudaGraphDestroy(got);
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return CDFCI_OK;
}

int build_block_graph(cdfci_ctx *c) {
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < c->mchunk && e == cudaSuccess; ++i) e = launch_mc_iteration(c->P, c->mb, c->stream);
    cudaGraph_t got = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &got);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (got) cudaGraphDestroy(got);
        return fail(CDFCI_ERR_CUDA, "capture of the multicoordinate iteration failed");
    }
    g = got;
    e = cudaGraphInstantiate(&c->mgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return CDFCI_OK;
}

// Candidate buffers (list, choice keys, tie scratch) of at least `need` entries: a start of more
// than m columns can touch more slots than one iteration.  The iteration graph holds the old
// buffers and Problem, so it is captured again.
int grow_candidates(cdfci_ctx *c, long long need) {
    McBuffers &b = c->mb;
    if (need <= b.cap_cand) return CDFCI_OK;
    long long *cand = nullptr;
    unsigned long long *gkey = nullptr;
    McSel *ties = nullptr;
    if (cudaMalloc(&cand, (size_t)need * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&gkey, (size_t)need * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&ties, (size_t)need * sizeof(McSel)) != cudaSuccess) {
        cudaFree(cand); cudaFree(gkey); cudaFree(ties);
        return fail(CDFCI_ERR_NOMEM, "candidate list of %lld entries does not fit", need);
    }
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < c->mb_nalloc; ++i) {
        void *&q = c->mb_alloc[i];
        if (q == (void *)b.cand) { cudaFree(q); q = cand; }
        else if (q == (void *)b.gkey) { cudaFree(q); q = gkey; }
        else if (q == (void *)b.ties) { cudaFree(q); q = ties; }
    }
    b.cand = cand;
    b.gkey = gkey;
    b.ties = ties;
    b.cap_cand = need;
    c->P.cap_cand = need;
    if (c->mgraph) {
        cudaGraphExecDestroy(c->mgraph);
        c->mgraph = nullptr;
    }
    return build_block_graph(c);
}

}  // namespace

namespace {
// Keys (2 words per entry) within N with the handle's electron counts, none repeated.
int check_keys(const cdfci_ctx *c, const std::vector<uint64_t> &k, int64_t n) {
    const unsigned long long full = c->N >= 64 ? ~0ull : ((1ull << c->N) - 1ull);
    std::vector<std::pair<uint64_t, uint64_t>> v((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t a = k[2 * i], b = k[2 * i + 1];
        if ((a & ~full) || (b & ~full) || __builtin_popcountll(a) != c->na || __builtin_popcountll(b) != c->nb)
            return fail(CDFCI_ERR_ARG, "entry %lld: key {%#llx, %#llx} does not match N = %d, n_alpha = %d, n_beta = %d",
                        (long long)i, (unsigned long long)a, (unsigned long long)b, c->N, c->na, c->nb);
        v[(size_t)i] = {a, b};
    }
    std::sort(v.begin(), v.end());
    for (size_t i = 1; i < v.size(); ++i)
        if (v[i] == v[i - 1])
            return fail(CDFCI_ERR_ARG, "key {%#llx, %#llx} appears twice", (unsigned long long)v[i].first,
                        (unsigned long long)v[i].second);
    return CDFCI_OK;
}

template <typename T>
int copy_in(std::vector<T> &dst, const T *src, size_t count) {
    dst.resize(count);
    if (count && cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDefault) != cudaSuccess)
        return fail(CDFCI_ERR_ARG, "input array could not be read (not host or device memory?)");
    return CDFCI_OK;
}

// Device copies of host arrays for one call; freed by the destructor.
struct DevTemp {
    std::vector<void *> p;
    template <typename T>
    T *put(const std::vector<T> &h, cudaStream_t s) {
        void *d = nullptr;
        if (cudaMalloc(&d, std::max<size_t>(h.size(), 1) * sizeof(T)) != cudaSuccess) return nullptr;
        p.push_back(d);
        if (!h.empty() && cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return nullptr;
        return static_cast<T *>(d);
    }
    template <typename T>
    T *alloc(size_t n) {
        void *d = nullptr;
        if (cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        p.push_back(d);
        return static_cast<T *>(d);
    }
    ~DevTemp() {
        for (void *d : p) cudaFree(d);
    }
};

// A fresh state word: no error, scale 1, zero counters.
int reset_state(cdfci_ctx *c) {
    IterState t;
    memset(&t, 0, sizeof(t));
    t.scale = dd_from(1.0);
    CK(cudaMemcpyAsync(c->d_st, &t, sizeof(t), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->d_table, 0, (size_t)c->P.capacity * sizeof(Slot), c->stream));
    if (c->block) CK(cudaMemsetAsync(c->mb.ms, 0, sizeof(McState), c->stream));
    if (c->P.cnz) CK(cudaMemsetAsync(c->P.cnz, 0, (size_t)(c->P.cnz_mask + 1) / 8, c->stream));
    if (c->P.mark) CK(cudaMemsetAsync(c->P.mark, 0, (size_t)((c->P.capacity + 31) / 32) * 4, c->stream));
    return CDFCI_OK;
}
}  // namespace

extern "C" {
#define CDFCI_API __attribute__((visibility("default")))

CDFCI_API void cdfci_default_params(cdfci_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->num_coordinates = 1;
    p->log2_capacity = 22;
    p->z_threshold = 0.0;
    p->max_load = 0.79;
    p->dx_damping = 0.9;
    p->dx_threshold = 0.0;
    p->deterministic = 1;
    p->num_states = 1;
    p->integral_symmetry = 8;
}

CDFCI_API const char *cdfci_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {
// cdfci_create, with the momentum tables of a k-space handle (host, ksub then kadd, N x N bytes
// each) or NULL.
int create_impl(const double *h, const double *g, int N, int n_alpha, int n_beta, const cdfci_params *params,
                const unsigned char *ktab, cdfci_handle *out) {
    if (!out) return fail(CDFCI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!h || !g) return fail(CDFCI_ERR_ARG, "h or g is NULL");
    if (N < 1 || N > kMaxN) return fail(CDFCI_ERR_ARG, "N = %d outside [1, %d]", N, kMaxN);
    if (n_alpha < 0 || n_beta < 0 || n_alpha > N || n_beta > N || n_alpha + n_beta == 0)
        return fail(CDFCI_ERR_ARG, "electron counts (%d, %d) invalid for N = %d", n_alpha, n_beta, N);
    cdfci_params prm;
    if (params) prm = *params; else cdfci_default_params(&prm);
    if (prm.num_coordinates < 1 || prm.num_coordinates > mc_max_m())
        return fail(CDFCI_ERR_ARG, "num_coordinates = %d outside [1, %d]", prm.num_coordinates, mc_max_m());
    if (prm.num_states == 0) prm.num_states = 1;
    if (prm.integral_symmetry == 0) prm.integral_symmetry = 8;
    if (prm.integral_symmetry != 8 && prm.integral_symmetry != 4)
        return fail(CDFCI_ERR_ARG, "integral_symmetry = %d (8 or 4)", prm.integral_symmetry);
    if (prm.num_states < 1 || prm.num_states > kXMax)
        return fail(CDFCI_ERR_ARG, "num_states = %d outside [1, %d]", prm.num_states, kXMax);
    if (prm.num_states > 1 && prm.num_coordinates != 1)
        return fail(CDFCI_ERR_ARG, "num_states = %d needs num_coordinates = 1 (Alg. 3 updates one row)", prm.num_states);
    if (!(prm.max_memory >= 0.0) || !std::isfinite(prm.max_memory)) return fail(CDFCI_ERR_ARG, "max_memory invalid");
    if (prm.max_memory > 0.0) {
        // the largest table whose slots (plus xCDFCI rows) fit in max_memory GiB
        const double per_slot = (double)sizeof(Slot) + (prm.num_states > 1 ? 16.0 * prm.num_states : 0.0);
        const double slots = prm.max_memory * 1073741824.0 / per_slot;
        int lc = 0;
        while (lc < 34 && std::ldexp(1.0, lc + 1) <= slots) ++lc;
        if (lc < 4) return fail(CDFCI_ERR_ARG, "max_memory = %g GiB holds fewer than 16 slots", prm.max_memory);
        prm.log2_capacity = lc;
    }
    if (prm.log2_capacity < 4 || prm.log2_capacity > 34)
        return fail(CDFCI_ERR_ARG, "log2_capacity = %d outside [4, 34]", prm.log2_capacity);
    if (!(prm.max_load > 0.0 && prm.max_load <= 0.95)) return fail(CDFCI_ERR_ARG, "max_load must be in (0, 0.95]");
    if (!(prm.z_threshold >= 0.0) || !std::isfinite(prm.z_threshold)) return fail(CDFCI_ERR_ARG, "z_threshold invalid");
    if (!(prm.dx_damping >= 0.0 && prm.dx_damping < 1.0)) return fail(CDFCI_ERR_ARG, "dx_damping must be in [0, 1)");
    unsigned long long refA = prm.ref_alpha, refB = prm.ref_beta;
    const unsigned long long full = N == 64 ? ~0ull : ((1ull << N) - 1ull);
    if (refA != 0ull || refB != 0ull) {
        if ((refA & ~full) || (refB & ~full) || __builtin_popcountll(refA) != n_alpha ||
            __builtin_popcountll(refB) != n_beta)
            return fail(CDFCI_ERR_ARG, "start determinant does not match N, n_alpha, n_beta");
    }

    cdfci_ctx *c = new (std::nothrow) cdfci_ctx();
    if (!c) return fail(CDFCI_ERR_NOMEM, "host allocation failed");
    c->prm = prm;
    c->N = N; c->na = n_alpha; c->nb = n_beta;
    int rc = CDFCI_OK;
    auto bail = [&](int code) { free_ctx(c); return code; };

    if (prm.cuda_stream) {
        c->stream = (cudaStream_t)prm.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(CDFCI_ERR_CUDA, "stream creation failed"));
        c->own_stream = true;
    }
    cudaStream_t s = c->stream;
    const size_t n2 = (size_t)N * N, n4 = n2 * n2;

    Problem &P = c->P;
    std::memset(&P, 0, sizeof(P));
    P.N = N; P.na = n_alpha; P.nb = n_beta; P.va = N - n_alpha; P.vb = N - n_beta;
    P.ca2 = (int)binom(P.na, 2); P.cb2 = (int)binom(P.nb, 2);
    P.cva2 = (int)binom(P.va, 2); P.cvb2 = (int)binom(P.vb, 2);
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
    P.capacity = 1ll << prm.log2_capacity;
    P.mask = (unsigned long long)P.capacity - 1ull;
    P.max_entries = (long long)std::floor(prm.max_load * (double)P.capacity);
    P.max_probe = (int)std::min<long long>(P.capacity, 1 << 16);
    P.tau = prm.z_threshold;
    P.theta = prm.dx_damping;
    P.dx_threshold = prm.dx_threshold;

    // integrals and derived tables
    if (cudaMalloc(&c->d_h, n2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_g, n4 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_J, n2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_K, n2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_W3, (size_t)N * n2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_V3, (size_t)N * n2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->d_flags, 4 * sizeof(int)) != cudaSuccess)
        return bail(fail(CDFCI_ERR_NOMEM, "device allocation of the integrals failed"));
    if (cudaMemcpyAsync(c->d_h, h, n2 * sizeof(double), kind_to_device(h), s) != cudaSuccess ||
        cudaMemcpyAsync(c->d_g, g, n4 * sizeof(double), kind_to_device(g), s) != cudaSuccess ||
        cudaMemsetAsync(c->d_flags, 0, 4 * sizeof(int), s) != cudaSuccess)
        return bail(fail(CDFCI_ERR_CUDA, "copy of the integrals failed"));
    if (launch_setup(c->d_h, c->d_g, N, c->d_J, c->d_K, c->d_W3, c->d_V3, c->d_flags, c->d_flags + 1,
                     prm.integral_symmetry == 4 ? 1 : 0, s) !=
        cudaSuccess)
        return bail(fail(CDFCI_ERR_CUDA, "set-up kernels failed to launch"));
    int flags[4];
    if (cudaMemcpyAsync(flags, c->d_flags, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return bail(fail(CDFCI_ERR_CUDA, "set-up failed"));
    if (flags[0] == CDFCI_ERR_NONFINITE) return bail(fail(CDFCI_ERR_NONFINITE, "h or g holds NaN/Inf"));
    if (flags[0] != 0)
        return bail(fail(CDFCI_ERR_ARG, "h is not symmetric or g lacks the %d-fold symmetry", prm.integral_symmetry));
    P.doubles_vanish = flags[1] ? 0 : 1;

    // pair tables: occupied alpha, occupied beta, virtual alpha, virtual beta
    std::vector<unsigned short> poa = pair_table(P.na), pob = pair_table(P.nb), pva = pair_table(P.va),
                                pvb = pair_table(P.vb);
    size_t npairs = poa.size() + pob.size() + pva.size() + pvb.size() + 1;
    std::vector<unsigned short> all;
    all.reserve(npairs);
    all.insert(all.end(), poa.begin(), poa.end());
    all.insert(all.end(), pob.begin(), pob.end());
    all.insert(all.end(), pva.begin(), pva.end());
    all.insert(all.end(), pvb.begin(), pvb.end());
    all.push_back(0);
    if (cudaMalloc(&c->d_pairs, all.size() * sizeof(unsigned short)) != cudaSuccess)
        return bail(fail(CDFCI_ERR_NOMEM, "device allocation failed"));
    if (cudaMemcpyAsync(c->d_pairs, all.data(), all.size() * sizeof(unsigned short), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return bail(fail(CDFCI_ERR_CUDA, "copy of pair tables failed"));
    P.pair_oa = c->d_pairs;
    P.pair_ob = P.pair_oa + poa.size();
    P.pair_va = P.pair_ob + pob.size();
    P.pair_vb = P.pair_va + pva.size();
    P.h = c->d_h; P.g = c->d_g; P.J = c->d_J; P.K = c->d_K; P.W3 = c->d_W3; P.V3 = c->d_V3;
    if (ktab) {
        if (cudaMalloc(&c->d_ktab, 2 * (size_t)N * N) != cudaSuccess)
            return bail(fail(CDFCI_ERR_NOMEM, "device allocation failed"));
        if (cudaMemcpyAsync(c->d_ktab, ktab, 2 * (size_t)N * N, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return bail(fail(CDFCI_ERR_CUDA, "copy of the momentum tables failed"));
        P.ksub = c->d_ktab;
        P.kadd = c->d_ktab + (size_t)N * N;
    }

    // table, state, partials, scratch
    if (cudaMalloc(&c->d_table, (size_t)P.capacity * sizeof(Slot)) != cudaSuccess)
        return bail(fail(CDFCI_ERR_NOMEM, "hash table of 2^%d slots (%.2f GiB) does not fit", prm.log2_capacity,
                         (double)P.capacity * sizeof(Slot) / (1 << 30)));
    P.table = c->d_table;
    {
        // About 256 column elements per CTA (0.73 per element thread): the loop is bound by the
        // latency of each element's dependent chain (generate, probe, update), not by bandwidth,
        // so spreading a column over more SMs pays until the per-iteration grid barrier dominates.
        // At most 64 CTAs by default: the control warp then folds every CTA's partial with one
        // round of loads (two per lane).
        const long long per_cta = 256;
        const long long nh_eff = P.doubles_vanish ? P.seg[2] : P.seg[5];
        const long long want = prm.grid_blocks > 0 ? prm.grid_blocks
                                                   : std::min<long long>((nh_eff - 1 + per_cta - 1) / per_cta, 64);
        const int maxg = want > 16 ? cd_max_grid(cd_dynamic_smem(P)) : 0;
        if (want > 16 && maxg > 16) {            // more CTAs than a cluster: the grid-wide loop
            c->gridmode = true;
            c->grid = (int)std::min<long long>(want, maxg);
        } else {
            c->grid = cd_pick_cluster((int)std::max<long long>(1, std::min<long long>(want, 16)), cd_dynamic_smem(P));
        }
    }
    // grid mode: after the G partials, the two exchange buffers of G x kXchgWords words (4 G CdPartials' worth)
    static_assert(2 * kXchgWords * sizeof(unsigned long long) == 4 * sizeof(CdPartial), "exchange buffer size");
    const size_t nparts = (size_t)c->grid * (c->gridmode ? 5 : 1);
    if (prm.graph_chunk > 0) c->chunk = prm.graph_chunk;
    if (cudaMemsetAsync(c->d_table, 0, (size_t)P.capacity * sizeof(Slot), s) != cudaSuccess ||
        cudaMalloc(&c->d_st, sizeof(IterState)) != cudaSuccess ||
        cudaMalloc(&c->d_part, nparts * sizeof(CdPartial)) != cudaSuccess ||
        cudaMalloc(&c->d_bar, sizeof(GridRound)) != cudaSuccess ||
        cudaMalloc(&c->d_rec, sizeof(CdRecord)) != cudaSuccess ||
        cudaMalloc(&c->d_counter, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_colkeys, (size_t)P.nh * 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&c->d_colvals, (size_t)P.nh * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&c->h_st, sizeof(IterState)) != cudaSuccess)
        return bail(fail(CDFCI_ERR_NOMEM, "device allocation failed"));
    if (cudaMemsetAsync(c->d_st, 0, sizeof(IterState), s) != cudaSuccess ||
        cudaMemsetAsync(c->d_rec, 0, sizeof(CdRecord), s) != cudaSuccess ||
        cudaMemsetAsync(c->d_part, 0, nparts * sizeof(CdPartial), s) != cudaSuccess ||
        cudaMemsetAsync(c->d_bar, 0, sizeof(GridRound), s) != cudaSuccess)
        return bail(fail(CDFCI_ERR_CUDA, "memset failed"));

    // start determinant: given, or aufbau on h_pp (smallest first, ties to the lower index)
    if (refA == 0ull && refB == 0ull) {
        std::vector<double> hd(n2);
        if (cudaMemcpyAsync(hd.data(), c->d_h, n2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return bail(fail(CDFCI_ERR_CUDA, "copy of h failed"));
        std::vector<int> order(N);
        for (int p = 0; p < N; ++p) order[p] = p;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return hd[(size_t)x * N + x] < hd[(size_t)y * N + y]; });
        for (int k = 0; k < n_alpha; ++k) refA |= 1ull << order[k];
        for (int k = 0; k < n_beta; ++k) refB |= 1ull << order[k];
    }
    if (prm.num_states > 1) {
        c->xcd = true;
        if (prm.graph_chunk > 0) c->mchunk = prm.graph_chunk;
        rc = setup_xcd(c, prm.num_states, refA, refB);
        if (rc != CDFCI_OK) return bail(rc);
        rc = fill_stats(c, nullptr);
        if (rc != CDFCI_OK) return bail(rc);
        rc = build_xcd_graph(c);
        if (rc != CDFCI_OK) return bail(rc);
        *out = c;
        return CDFCI_OK;
    }
    if (prm.num_coordinates > 1) {
        c->block = true;
        rc = setup_block(c, prm.num_coordinates);
        if (rc != CDFCI_OK) return bail(rc);
        if (prm.graph_chunk > 0) c->mchunk = prm.graph_chunk;
        // start vector c = e_ref, b = H e_ref (compression applied): first column with eta = 1
        if (launch_mc_start(P, c->mb, refA, refB, 1.0, 1, s) != cudaSuccess ||
            launch_mc_scatter_finalize(P, c->mb, s) != cudaSuccess)
            return bail(fail(CDFCI_ERR_CUDA, "initial column launch failed"));
        rc = fill_stats(c, nullptr);
        if (rc != CDFCI_OK) return bail(rc);
        rc = build_block_graph(c);
        if (rc != CDFCI_OK) return bail(rc);
        *out = c;
        return CDFCI_OK;
    }
    if (launch_init_state(c->d_st, c->d_rec, refA, refB, 1.0, s) != cudaSuccess)
        return bail(fail(CDFCI_ERR_CUDA, "init launch failed"));
    // initialisation iteration: c = e_ref, b = H e_ref (compression applied)
    rc = run_iterations(c, 1);
    if (rc != CDFCI_OK) return bail(rc);
    rc = fill_stats(c, nullptr);
    if (rc != CDFCI_OK) return bail(rc);
    *out = c;
    return CDFCI_OK;
}
}  // namespace

extern "C" {

CDFCI_API int cdfci_create(const double *h, const double *g, int N, int n_alpha, int n_beta, const cdfci_params *params,
                 cdfci_handle *out) {
    return create_impl(h, g, N, n_alpha, n_beta, params, nullptr, out);
}

CDFCI_API int cdfci_create_hubbard_k(const int32_t *shape, int32_t D, double t, double U, int n_alpha, int n_beta,
                                     const cdfci_params *params, cdfci_handle *out) {
    if (!out) return fail(CDFCI_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!shape || D < 1 || D > 8) return fail(CDFCI_ERR_ARG, "lattice dimension D = %d outside [1, 8]", (int)D);
    long long L = 1;
    for (int d = 0; d < D; ++d) {
        if (shape[d] < 1) return fail(CDFCI_ERR_ARG, "extent %d of direction %d", (int)shape[d], d);
        L *= shape[d];
        if (L > kMaxN) return fail(CDFCI_ERR_ARG, "%lld sites exceed %d orbitals", L, kMaxN);
    }
    if (!std::isfinite(t) || !std::isfinite(U)) return fail(CDFCI_ERR_ARG, "t or U is not finite");
    const int N = (int)L;
    // momentum indices n_p, row-major (the last direction fastest)
    std::vector<int> mom((size_t)N * D);
    for (int p = 0; p < N; ++p) {
        int r = p;
        for (int d = D - 1; d >= 0; --d) { mom[(size_t)p * D + d] = r % shape[d]; r /= shape[d]; }
    }
    auto index_of = [&](const int *m) {
        int p = 0;
        for (int d = 0; d < D; ++d) p = p * shape[d] + (((m[d] % shape[d]) + shape[d]) % shape[d]);
        return p;
    };
    // eps_k of the nearest-neighbour hopping: -2t cos k_d per direction of extent >= 3 (two bonds),
    // -t cos k_d for extent 2 (one bond), none for extent 1; rounded to 12 decimals
    std::vector<double> h((size_t)N * N, 0.0);
    for (int p = 0; p < N; ++p) {
        double e = 0.0;
        for (int d = 0; d < D; ++d) {
            const double k = 2.0 * M_PI * mom[(size_t)p * D + d] / shape[d];
            if (shape[d] >= 3) e += -2.0 * t * std::cos(k);
            else if (shape[d] == 2) e += -t * std::cos(k);
        }
        h[(size_t)p * N + p] = std::nearbyint(e * 1e12) / 1e12 + 0.0;
    }
    // (pq|rs) = U/L when k_q - k_p + k_s - k_r = 0; momentum tables
    std::vector<unsigned char> ktab(2 * (size_t)N * N);
    std::vector<int> m(D);
    for (int p = 0; p < N; ++p)
        for (int q = 0; q < N; ++q) {
            for (int d = 0; d < D; ++d) m[d] = mom[(size_t)q * D + d] - mom[(size_t)p * D + d];
            ktab[(size_t)p * N + q] = (unsigned char)index_of(m.data());
            for (int d = 0; d < D; ++d) m[d] = mom[(size_t)p * D + d] + mom[(size_t)q * D + d];
            ktab[(size_t)N * N + (size_t)p * N + q] = (unsigned char)index_of(m.data());
        }
    std::vector<double> g((size_t)N * N * N * N, 0.0);
    const double v = U / (double)N;
    for (int p = 0; p < N; ++p)
        for (int q = 0; q < N; ++q)
            for (int r = 0; r < N; ++r)
                for (int s2 = 0; s2 < N; ++s2)
                    if (ktab[(size_t)N * N + (size_t)ktab[(size_t)p * N + q] * N + ktab[(size_t)r * N + s2]] == 0)
                        g[(((size_t)p * N + q) * N + r) * N + s2] = v;
    cdfci_params prm;
    if (params) prm = *params; else cdfci_default_params(&prm);
    prm.integral_symmetry = 4;
    return create_impl(h.data(), g.data(), N, n_alpha, n_beta, &prm, ktab.data(), out);
}

CDFCI_API int cdfci_step(cdfci_handle c, int64_t n_iter, cdfci_stats *stats) {
    if (!c) return fail(CDFCI_ERR_ARG, "handle is NULL");
    if (n_iter < 0) return fail(CDFCI_ERR_ARG, "n_iter < 0");
    if (c->block || c->xcd) {
        for (int64_t i = 0; i < n_iter / c->mchunk; ++i) {
            bool changed = false;
            int rc = maybe_raise_tau(c, &changed);
            if (rc) return rc;
            if (changed) {                                       // tau is a launch parameter of the graph
                cudaGraphExecDestroy(c->mgraph);
                c->mgraph = nullptr;
                rc = c->xcd ? build_xcd_graph(c) : build_block_graph(c);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(c->mgraph, c->stream));
        }
        for (int64_t i = 0; i < n_iter % c->mchunk; ++i)
            CK(c->xcd ? launch_x_iteration(c->P, c->xb, c->stream) : launch_mc_iteration(c->P, c->mb, c->stream));
        return fill_stats(c, stats);
    }
    int rc = run_iterations(c, n_iter);
    if (rc) return rc;
    return fill_stats(c, stats);
}

CDFCI_API int cdfci_get_stats(cdfci_handle c, cdfci_stats *stats) {
    if (!c) return fail(CDFCI_ERR_ARG, "handle is NULL");
    return fill_stats(c, stats);
}

CDFCI_API int cdfci_energy(cdfci_handle c, int mode, double *E) {
    if (!c || !E) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (mode == 0) {
        int rc = fill_stats(c, nullptr);
        if (rc) return rc;
        *E = c->h_st->energy;
        return CDFCI_OK;
    }
    if (mode != 1) return fail(CDFCI_ERR_ARG, "mode must be 0 or 1");
    if (c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "exact recompute (mode 1) is for one state; use cdfci_energies");
    int rc = fill_stats(c, nullptr);
    if (rc) return rc;
    return exact_rq(c, c->P, E);
}

CDFCI_API int cdfci_energy_with(cdfci_handle c, const double *h, const double *g, double *E) {
    if (!c || !h || !g || !E) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "the Rayleigh quotient under other integrals is for one state");
    int rc = fill_stats(c, nullptr);
    if (rc) return rc;
    const int N = c->N;
    const size_t n2 = (size_t)N * N, n4 = n2 * n2;
    double *dh = nullptr, *dg = nullptr, *dJ = nullptr, *dK = nullptr, *dW3 = nullptr, *dV3 = nullptr;
    int *dflags = nullptr;
    auto release = [&]() {
        cudaFree(dh); cudaFree(dg); cudaFree(dJ); cudaFree(dK); cudaFree(dW3); cudaFree(dV3); cudaFree(dflags);
    };
    if (cudaMalloc(&dh, n2 * sizeof(double)) != cudaSuccess || cudaMalloc(&dg, n4 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dJ, n2 * sizeof(double)) != cudaSuccess || cudaMalloc(&dK, n2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dW3, (size_t)N * n2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dV3, (size_t)N * n2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dflags, 4 * sizeof(int)) != cudaSuccess) {
        release();
        return fail(CDFCI_ERR_NOMEM, "device allocation of the integrals failed");
    }
    int flags[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(dh, h, n2 * sizeof(double), kind_to_device(h), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dg, g, n4 * sizeof(double), kind_to_device(g), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dflags, 0, 4 * sizeof(int), c->stream);
    if (e == cudaSuccess)
        e = launch_setup(dh, dg, N, dJ, dK, dW3, dV3, dflags, dflags + 1, c->prm.integral_symmetry == 4 ? 1 : 0,
                         c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags, dflags, sizeof(flags), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { release(); return fail(CDFCI_ERR_CUDA, "set-up of the integrals: %s", cudaGetErrorString(e)); }
    if (flags[0] == CDFCI_ERR_NONFINITE) { release(); return fail(CDFCI_ERR_NONFINITE, "h or g holds NaN/Inf"); }
    if (flags[0] != 0) {
        release();
        return fail(CDFCI_ERR_ARG, "h is not symmetric or g lacks the %d-fold symmetry", c->prm.integral_symmetry);
    }
    Problem P = c->P;
    P.h = dh; P.g = dg; P.J = dJ; P.K = dK; P.W3 = dW3; P.V3 = dV3;
    P.doubles_vanish = flags[1] ? 0 : 1;
    rc = exact_rq(c, P, E);
    release();
    return rc;
}

}  // extern "C"

namespace {
// c^T H c / c^T c of the handle's stored vector with H from P's integrals: every stored i with
// c_i != 0 gets (Hc)_i from a fresh column (lookups only), partial sums reduced in a fixed order.
int exact_rq(cdfci_ctx *c, const Problem &P, double *E) {
    long long n = c->h_st->n_slots;
    long long *list = nullptr;
    double *partial = nullptr, *dE = nullptr;
    const int nblocks = 152 * 4;
    if (cudaMalloc(&list, (size_t)std::max<long long>(n, 1) * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&partial, (size_t)nblocks * 2 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dE, sizeof(double)) != cudaSuccess) {
        cudaFree(list); cudaFree(partial); cudaFree(dE);
        return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    }
    cudaError_t e = cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = launch_rq(P, c->d_st, list, n, c->d_counter, partial, nblocks, dE, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E, dE, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(list); cudaFree(partial); cudaFree(dE);
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "energy: %s", cudaGetErrorString(e));
    return fill_stats(c, nullptr);
}
}  // namespace

extern "C" {

CDFCI_API int cdfci_get_column(cdfci_handle c, const uint64_t *key, uint64_t *keys_out, double *vals_out, int64_t cap,
                     int64_t *n_out) {
    if (!c || !key || !n_out) return fail(CDFCI_ERR_ARG, "NULL argument");
    uint64_t k[2];
    if (is_device_ptr(key)) {
        CK(cudaMemcpy(k, key, sizeof(k), cudaMemcpyDeviceToHost));
    } else {
        k[0] = key[0]; k[1] = key[1];
    }
    const unsigned long long full = (1ull << c->N) - 1ull;
    if ((k[0] & ~full) || (k[1] & ~full) || __builtin_popcountll(k[0]) != c->na || __builtin_popcountll(k[1]) != c->nb)
        return fail(CDFCI_ERR_ARG, "key does not match N, n_alpha, n_beta");
    CK(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream));
    CK(launch_column(c->P, k[0], k[1], c->d_colkeys, c->d_colvals, c->P.nh, c->d_counter, c->stream));
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, c->d_counter, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *n_out = (int64_t)n;
    if ((int64_t)n > cap) return fail(CDFCI_ERR_CAPACITY, "column has %lld entries, cap is %lld", (long long)n, (long long)cap);
    if (n > 0) {
        if (keys_out)
            CK(cudaMemcpyAsync(keys_out, c->d_colkeys, n * 2 * sizeof(uint64_t), cudaMemcpyDefault, c->stream));
        if (vals_out) CK(cudaMemcpyAsync(vals_out, c->d_colvals, n * sizeof(double), cudaMemcpyDefault, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return CDFCI_OK;
}

CDFCI_API int cdfci_get_entry(cdfci_handle c, const uint64_t *row_key, const uint64_t *col_key, double *value) {
    if (!c || !row_key || !col_key || !value) return fail(CDFCI_ERR_ARG, "NULL argument");
    uint64_t k[4];
    for (int t = 0; t < 2; ++t) {
        const uint64_t *src = t == 0 ? row_key : col_key;
        if (is_device_ptr(src)) {
            CK(cudaMemcpy(k + 2 * t, src, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        } else {
            k[2 * t] = src[0];
            k[2 * t + 1] = src[1];
        }
    }
    const unsigned long long full = c->N >= 64 ? ~0ull : ((1ull << c->N) - 1ull);
    for (int t = 0; t < 2; ++t)
        if ((k[2 * t] & ~full) || (k[2 * t + 1] & ~full) || __builtin_popcountll(k[2 * t]) != c->na ||
            __builtin_popcountll(k[2 * t + 1]) != c->nb)
            return fail(CDFCI_ERR_ARG, "key does not match N, n_alpha, n_beta");
    DevTemp tmp;
    double *d = tmp.put(std::vector<double>(1, 0.0), c->stream);
    if (!d) return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    CK(launch_entry(c->P, k[0], k[1], k[2], k[3], d, c->stream));
    CK(cudaMemcpyAsync(value, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return CDFCI_OK;
}

CDFCI_API int cdfci_get_diagonal(cdfci_handle c, const uint64_t *key, double *value) {
    return cdfci_get_entry(c, key, key, value);
}

CDFCI_API int cdfci_optorb(const double *h, const double *g, int M, int N, int n_alpha, int n_beta, double *U,
                           const cdfci_optorb_params *p, double *energies) {
    if (!h || !g || !U || !p || !energies) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (M < 1 || M > kMaxN || N < 1 || N > M) return fail(CDFCI_ERR_ARG, "need 1 <= N <= M <= %d", kMaxN);
    if (p->outer < 1 || p->bb_steps < 0 || p->inner_iterations < 0)
        return fail(CDFCI_ERR_ARG, "outer >= 1, bb_steps >= 0 and inner_iterations >= 0 required");
    if (p->fci.num_states > 1) return fail(CDFCI_ERR_ARG, "the inner FCI solves one state (num_states = 1)");
    const long long MN = (long long)M * N, M2 = (long long)M * M, N2 = (long long)N * N;
    const long long M4 = M2 * M2, N3 = N2 * N, N4 = N2 * N2;
    std::vector<double> hU0;
    int rc = copy_in(hU0, U, (size_t)MN);
    if (rc) return rc;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            double x = 0.0;
            for (int q = 0; q < M; ++q) x += hU0[(size_t)q * N + a] * hU0[(size_t)q * N + b];
            if (std::fabs(x - (a == b ? 1.0 : 0.0)) > 1e-10) return fail(CDFCI_ERR_ARG, "U has no orthonormal columns");
        }
    cudaStream_t s = nullptr;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard { cudaStream_t s; ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); } } sg{s};
    DevTemp tmp;
    double *dh = tmp.alloc<double>(M2), *dg = tmp.alloc<double>(M4), *dU = tmp.alloc<double>(MN);
    double *t1 = tmp.alloc<double>(M2 * M * N), *t2 = tmp.alloc<double>(M2 * N2), *g3 = tmp.alloc<double>(M * N3);
    double *g4 = tmp.alloc<double>(N4), *hU = tmp.alloc<double>(MN), *h2 = tmp.alloc<double>(N2);
    double *r1 = tmp.alloc<double>(N2), *r2 = tmp.alloc<double>(N4), *G = tmp.alloc<double>(MN);
    double *Uo = tmp.alloc<double>(MN), *Go = tmp.alloc<double>(MN), *X = tmp.alloc<double>(MN);
    double *Xn = tmp.alloc<double>(MN), *Gm = tmp.alloc<double>(N2), *Ub = tmp.alloc<double>(MN);
    double *sc = tmp.alloc<double>(8);
    if (!dh || !dg || !dU || !t1 || !t2 || !g3 || !g4 || !hU || !h2 || !r1 || !r2 || !G || !Uo || !Go || !X || !Xn ||
        !Gm || !Ub || !sc)
        return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    CK(cudaMemcpyAsync(dh, h, M2 * sizeof(double), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(dg, g, M4 * sizeof(double), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(dU, hU0.data(), MN * sizeof(double), cudaMemcpyHostToDevice, s));
    const size_t bMN = MN * sizeof(double);
    // h' = U^T h U, g' (all four indices), and g'' (three) for the gradient
    auto transform = [&](const double *Uc) -> cudaError_t {
        cudaError_t e = oo_contract(dg, Uc, t1, M2 * M, M, N, 1, s);
        if (e == cudaSuccess) e = oo_contract(t1, Uc, t2, M2, M, N, N, s);
        if (e == cudaSuccess) e = oo_contract(t2, Uc, g3, M, M, N, N2, s);
        if (e == cudaSuccess) e = oo_contract(g3, Uc, g4, 1, M, N, N3, s);
        if (e == cudaSuccess) e = oo_contract(dh, Uc, hU, M, M, N, 1, s);
        if (e == cudaSuccess) e = oo_contract(hU, Uc, h2, 1, M, N, N, s);
        return e;
    };
    auto read = [&](int k, double *out) -> int {
        CK(cudaMemcpyAsync(out, sc, k * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return CDFCI_OK;
    };
    auto objective = [&](double *P) -> int {                       // P4 from h', g' and the RDMs
        CK(oo_dot(h2, r1, N2, sc, s));
        CK(oo_dot(g4, r2, N4, sc + 1, s));
        double v[2];
        int r = read(2, v);
        *P = v[0] + 0.5 * v[1];
        return r;
    };
    auto polar = [&]() -> int {                                    // X <- orth(X) (Newton-Schulz on X / ||X||_F)
        CK(oo_dot(X, X, MN, sc, s));
        CK(oo_scale(X, sc, MN, s));
        std::vector<double> gm((size_t)N2);
        for (int k = 0; k < 200; ++k) {
            CK(oo_gram(X, Gm, M, N, s));
            CK(cudaMemcpyAsync(gm.data(), Gm, N2 * sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            double err = 0.0;
            for (int a = 0; a < N; ++a)
                for (int b = 0; b < N; ++b) err = std::max(err, std::fabs(gm[(size_t)a * N + b] - (a == b ? 1.0 : 0.0)));
            if (err < 4e-16 * N) return CDFCI_OK;
            CK(oo_ns(X, Gm, Xn, M, N, s));
            std::swap(X, Xn);
        }
        return fail(CDFCI_ERR_INTERNAL, "the orthogonal projection did not converge");
    };
    for (int it = 0; it < p->outer; ++it) {
        CK(transform(dU));
        cdfci_params fp = p->fci;
        fp.cuda_stream = s;
        cdfci_handle hd = nullptr;
        rc = cdfci_create(h2, g4, N, n_alpha, n_beta, &fp, &hd);
        if (rc) return rc;
        cdfci_stats st;
        rc = cdfci_step(hd, p->inner_iterations, &st);
        if (!rc) rc = cdfci_rdm(hd, r1, r2);
        cdfci_destroy(hd);
        if (rc) return rc;
        energies[it] = st.energy;
        // the orbital subproblem with these RDMs
        double P = 0.0, best = 0.0;
        if ((rc = objective(&P))) return rc;
        best = P;
        CK(cudaMemcpyAsync(Ub, dU, bMN, cudaMemcpyDeviceToDevice, s));
        CK(oo_grad(hU, r1, g3, r2, G, M, N, s));
        CK(oo_dot(G, G, MN, sc, s));
        double gg = 0.0;
        if ((rc = read(1, &gg))) return rc;
        double t = 0.1 / std::max(1.0, std::sqrt(gg));
        for (int k = 0; k < p->bb_steps; ++k) {
            if (k > 0) {
                CK(oo_axpy(dU, Uo, 1.0, X, MN, s));                  // S = U - U_old
                CK(oo_axpy(G, Go, 1.0, Xn, MN, s));                  // Y = G - G_old
                CK(oo_dot(X, X, MN, sc, s));
                CK(oo_dot(X, Xn, MN, sc + 1, s));
                CK(oo_dot(Xn, Xn, MN, sc + 2, s));
                double d[3];
                if ((rc = read(3, d))) return rc;
                if (std::fabs(d[1]) > 0.0 && d[2] > 0.0) t = (k % 2 == 1) ? d[0] / std::fabs(d[1]) : std::fabs(d[1]) / d[2];
                t = std::min(std::max(t, 1e-10), 1e10);
            }
            CK(cudaMemcpyAsync(Uo, dU, bMN, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(Go, G, bMN, cudaMemcpyDeviceToDevice, s));
            CK(oo_axpy(dU, G, t, X, MN, s));                         // X = U - t grad
            if ((rc = polar())) return rc;
            CK(cudaMemcpyAsync(dU, X, bMN, cudaMemcpyDeviceToDevice, s));
            CK(transform(dU));
            CK(oo_grad(hU, r1, g3, r2, G, M, N, s));
            if ((rc = objective(&P))) return rc;
            if (P < best) {
                best = P;
                CK(cudaMemcpyAsync(Ub, dU, bMN, cudaMemcpyDeviceToDevice, s));
            }
        }
        CK(cudaMemcpyAsync(dU, Ub, bMN, cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaMemcpyAsync(U, dU, bMN, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return CDFCI_OK;
}

CDFCI_API int cdfci_energies(cdfci_handle c, double *E, int32_t cap, int32_t *n_out) {
    if (!c || !E || !n_out) return fail(CDFCI_ERR_ARG, "NULL argument");
    int rc = fill_stats(c, nullptr);
    if (rc) return rc;
    *n_out = c->k1;
    if (cap < c->k1) return fail(CDFCI_ERR_CAPACITY, "%d energies, cap is %d", c->k1, (int)cap);
    if (!c->xcd) {
        E[0] = c->h_st->energy;
        return CDFCI_OK;
    }
    XState x;
    CK(cudaMemcpy(&x, c->xb.xs, sizeof(x), cudaMemcpyDeviceToHost));
    for (int a = 0; a < c->k1; ++a) E[a] = x.E[a];
    return CDFCI_OK;
}

}  // extern "C"

namespace {
// The strings of ne electrons with the lowest one-body energy: the shells below
// the ne-th level filled, every choice of the rest in the last shell.
std::vector<uint64_t> lowest_strings(const std::vector<double> &eps, int ne, double tol, int64_t cap, bool &over) {
    const int N = (int)eps.size();
    std::vector<uint64_t> out;
    over = false;
    if (ne == 0) { out.push_back(0); return out; }
    std::vector<int> order(N);
    for (int p = 0; p < N; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return eps[x] < eps[y]; });
    const double top = eps[order[ne - 1]], band = tol * std::max(1.0, std::fabs(top));
    uint64_t below = 0;
    std::vector<int> shell;
    for (int p = 0; p < N; ++p) {
        if (eps[p] < top - band) below |= 1ull << p;
        else if (eps[p] <= top + band) shell.push_back(p);
    }
    const int r = ne - __builtin_popcountll(below);
    // C(|shell|, r) choices, bounded before they are listed
    double count = 1.0;
    for (int k = 0; k < r; ++k) count = count * (double)(shell.size() - k) / (double)(k + 1);
    if (count > (double)cap) { over = true; return out; }
    std::vector<int> pick(r);
    for (int k = 0; k < r; ++k) pick[k] = k;
    while (true) {
        uint64_t m = below;
        for (int k = 0; k < r; ++k) m |= 1ull << shell[pick[k]];
        out.push_back(m);
        int k = r - 1;
        while (k >= 0 && pick[k] == (int)shell.size() - r + k) --k;
        if (k < 0) break;
        ++pick[k];
        for (int j = k + 1; j < r; ++j) pick[j] = pick[j - 1] + 1;
    }
    return out;
}

// The degenerate set S = alpha choices x beta choices, ordered by the 128-bit key; *n_det = |S|
// (cap + 1 when a spin's choices alone exceed cap).
int degenerate_configurations(const std::vector<double> &eps, int na, int nb, double tol, int64_t cap,
                              std::vector<std::pair<uint64_t, uint64_t>> &S, int64_t *n_det) {
    bool overA = false, overB = false;
    const std::vector<uint64_t> sa = lowest_strings(eps, na, tol, cap, overA), sb = lowest_strings(eps, nb, tol, cap, overB);
    const double total = (double)sa.size() * (double)sb.size();
    if (overA || overB || total > (double)cap) {
        *n_det = (overA || overB) ? cap + 1 : (int64_t)total;
        return fail(CDFCI_ERR_CAPACITY, "the degenerate set exceeds cap = %lld", (long long)cap);
    }
    S.clear();
    for (uint64_t b : sb)
        for (uint64_t a : sa) S.push_back({b, a});
    std::sort(S.begin(), S.end());
    *n_det = (int64_t)S.size();
    return CDFCI_OK;
}

// The start vector of the degenerate subspace: the eigenpairs of the symmetric
// n x n matrix A (row-major, destroyed) by cyclic Jacobi rotations (each zeroes
// A_pq with tan = t, t the smaller root of t^2 + 2 theta t - 1 = 0, theta =
// (A_qq - A_pp) / (2 A_pq)); lam = the lowest eigenvalue; v = the projection
// onto its whole eigenspace (eigenvalues within 1e-9 of it, relative) of the
// ramp r_s = 1 + s / n, normalised with its largest component positive (ties:
// the first).  For a simple eigenvalue v is its eigenvector; for a degenerate
// one the projection has a component in every momentum sector of the
// eigenspace, where a single basis vector may lie in one sector only.
void jacobi_lowest(int n, std::vector<double> &A, double &lam, std::vector<double> &v) {
    std::vector<double> V((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double norm2 = 0.0;
    for (double x : A) norm2 += x * x;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (off <= 1e-32 * norm2 || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {               // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = cs * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {               // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = cs * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = cs * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    int lo = 0;
    for (int i = 1; i < n; ++i)
        if (A[(size_t)i * n + i] < A[(size_t)lo * n + lo]) lo = i;
    lam = A[(size_t)lo * n + lo];
    const double band = 1e-9 * std::max(1.0, std::fabs(lam));
    v.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        if (!(A[(size_t)j * n + j] <= lam + band)) continue;
        double dot = 0.0;                                   // (eigenvector j) . ramp
        for (int k = 0; k < n; ++k) dot += V[(size_t)k * n + j] * (1.0 + (double)k / (double)n);
        for (int k = 0; k < n; ++k) v[k] += dot * V[(size_t)k * n + j];
    }
    double nrm = 0.0;
    for (int k = 0; k < n; ++k) nrm += v[k] * v[k];
    nrm = std::sqrt(nrm);
    int big = 0;
    for (int k = 0; k < n; ++k) {
        v[k] /= nrm;
        if (std::fabs(v[k]) > std::fabs(v[big])) big = k;
    }
    if (v[big] < 0.0)
        for (double &x : v) x = -x;
}
}  // namespace

extern "C" {

CDFCI_API int cdfci_degenerate_set(const double *eps, int N, int n_alpha, int n_beta, double tol, int64_t cap,
                                   uint64_t *keys, int64_t *n_det) {
    if (!eps || !n_det) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (N < 1 || N > kMaxN) return fail(CDFCI_ERR_ARG, "N = %d outside [1, %d]", N, kMaxN);
    if (n_alpha < 0 || n_beta < 0 || n_alpha > N || n_beta > N)
        return fail(CDFCI_ERR_ARG, "electron counts (%d, %d) invalid for N = %d", n_alpha, n_beta, N);
    if (!(tol > 0.0)) tol = 1e-10;
    if (keys && cap <= 0) return fail(CDFCI_ERR_ARG, "cap must be > 0 when keys is given");
    if (cap <= 0) cap = 1024;
    std::vector<double> e(eps, eps + N);
    for (double x : e)
        if (!std::isfinite(x)) return fail(CDFCI_ERR_ARG, "a one-body level is not finite");
    std::vector<std::pair<uint64_t, uint64_t>> S;
    const int rc = degenerate_configurations(e, n_alpha, n_beta, tol, cap, S, n_det);
    if (rc) return rc;
    if (keys)
        for (size_t i = 0; i < S.size(); ++i) {
            keys[2 * i] = S[i].second;
            keys[2 * i + 1] = S[i].first;
        }
    return CDFCI_OK;
}

CDFCI_API int cdfci_set_initial_degenerate(cdfci_handle c, double tol, int64_t cap, int64_t *n_det, double *E_sub) {
    if (!c || !n_det) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "start vectors are for one state (num_states = 1)");
    if (!(tol > 0.0)) tol = 1e-10;
    if (cap <= 0) cap = 1024;
    const int N = c->N;
    std::vector<double> hd((size_t)N * N);
    CK(cudaMemcpy(hd.data(), c->d_h, hd.size() * sizeof(double), cudaMemcpyDeviceToHost));
    std::vector<double> eps(N);
    for (int p = 0; p < N; ++p) eps[p] = hd[(size_t)p * N + p];
    std::vector<std::pair<uint64_t, uint64_t>> S;                // (B, A): the 128-bit key order
    int rc = degenerate_configurations(eps, c->na, c->nb, tol, cap, S, n_det);
    if (rc) return rc;
    const int n = (int)S.size();
    std::map<std::pair<uint64_t, uint64_t>, int> index;
    for (int i = 0; i < n; ++i) index[S[i]] = i;
    // H_SS from the columns: column i holds H_{D', D_i}
    std::vector<double> H((size_t)n * n, 0.0);
    std::vector<uint64_t> ck((size_t)c->P.nh * 2);
    std::vector<double> cv((size_t)c->P.nh);
    for (int i = 0; i < n; ++i) {
        CK(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream));
        CK(launch_column(c->P, S[i].second, S[i].first, c->d_colkeys, c->d_colvals, c->P.nh, c->d_counter, c->stream));
        unsigned long long cnt = 0;
        CK(cudaMemcpyAsync(&cnt, c->d_counter, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if ((long long)cnt > c->P.nh) return fail(CDFCI_ERR_INTERNAL, "column longer than its enumeration");
        if (cnt > 0) {
            CK(cudaMemcpyAsync(ck.data(), c->d_colkeys, cnt * 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(cv.data(), c->d_colvals, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
        for (unsigned long long e = 0; e < cnt; ++e) {
            const auto it = index.find({ck[2 * e + 1], ck[2 * e]});
            if (it != index.end()) H[(size_t)it->second * n + i] = cv[e];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double x = 0.5 * (H[(size_t)i * n + j] + H[(size_t)j * n + i]);
            H[(size_t)i * n + j] = H[(size_t)j * n + i] = x;
        }
    double lam = 0.0;
    std::vector<double> v;
    jacobi_lowest(n, H, lam, v);
    if (E_sub) *E_sub = lam;
    std::vector<uint64_t> keys;
    std::vector<double> cvals;
    for (int i = 0; i < n; ++i)
        if (v[i] != 0.0) {
            keys.push_back(S[i].second);
            keys.push_back(S[i].first);
            cvals.push_back(v[i]);
        }
    return cdfci_set_initial(c, keys.data(), cvals.data(), (int64_t)cvals.size());
}

CDFCI_API int cdfci_time_kernels(cdfci_handle c, int64_t n_iter, double *ms, int32_t cap, int32_t *n_kernels) {
    if (!c || !ms || !n_kernels) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (n_iter < 0) return fail(CDFCI_ERR_ARG, "n_iter < 0");
    if (!c->block || c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "per-kernel times are for mCDFCI handles");
    *n_kernels = kMcKernels;
    if (cap < kMcKernels) return fail(CDFCI_ERR_CAPACITY, "%d kernels, cap is %d", kMcKernels, (int)cap);
    for (int k = 0; k < kMcKernels; ++k) ms[k] = 0.0;
    cudaEvent_t ev[kMcKernels + 1];
    int made = 0;
    for (; made <= kMcKernels; ++made)
        if (cudaEventCreate(&ev[made]) != cudaSuccess) break;
    int rc = made <= kMcKernels ? fail(CDFCI_ERR_CUDA, "cudaEventCreate failed") : CDFCI_OK;
    for (int64_t i = 0; i < n_iter && rc == CDFCI_OK; ++i) {
        if (launch_mc_iteration(c->P, c->mb, c->stream, ev) != cudaSuccess ||
            cudaEventSynchronize(ev[kMcKernels]) != cudaSuccess) {
            rc = fail(CDFCI_ERR_CUDA, "timed iteration failed");
            break;
        }
        for (int k = 0; k < kMcKernels; ++k) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, ev[k], ev[k + 1]) != cudaSuccess) { rc = fail(CDFCI_ERR_CUDA, "event timing failed"); break; }
            ms[k] += t;
        }
    }
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    if (rc != CDFCI_OK) return rc;
    return fill_stats(c, nullptr);
}

CDFCI_API int cdfci_export_states(cdfci_handle c, uint64_t *keys, double *C, double *B, int64_t cap,
                                  int64_t *n_out) {
    if (!c || !n_out) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (!c->xcd) return cdfci_export(c, keys, C, B, cap, n_out);
    int rc = fill_stats(c, nullptr);
    if (rc) return rc;
    const long long n = c->h_st->n_slots, k1 = c->k1;
    *n_out = n;
    if (n > cap) return fail(CDFCI_ERR_CAPACITY, "%lld entries stored, cap is %lld", n, (long long)cap);
    if (n == 0) return CDFCI_OK;
    unsigned long long *dk = nullptr;
    double *dc = nullptr, *db = nullptr;
    if (cudaMalloc(&dk, (size_t)n * 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&dc, (size_t)n * k1 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&db, (size_t)n * k1 * sizeof(double)) != cudaSuccess) {
        cudaFree(dk); cudaFree(dc); cudaFree(db);
        return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    }
    cudaError_t e = cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = launch_x_export(c->P, c->xb, c->k1, dk, dc, db, n, c->d_counter, c->stream);
    if (e == cudaSuccess && keys) e = cudaMemcpyAsync(keys, dk, (size_t)n * 2 * sizeof(uint64_t), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && C) e = cudaMemcpyAsync(C, dc, (size_t)n * k1 * sizeof(double), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && B) e = cudaMemcpyAsync(B, db, (size_t)n * k1 * sizeof(double), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(dk); cudaFree(dc); cudaFree(db);
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "export_states: %s", cudaGetErrorString(e));
    return CDFCI_OK;
}

CDFCI_API int cdfci_export(cdfci_handle c, uint64_t *keys, double *cv, double *bv, int64_t cap, int64_t *n_out) {
    if (!c || !n_out) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "a num_states > 1 handle stores rows: use cdfci_export_states");
    int rc = fill_stats(c, nullptr);
    if (rc) return rc;
    long long n = c->h_st->n_slots;
    *n_out = n;
    if (n > cap) return fail(CDFCI_ERR_CAPACITY, "%lld entries stored, cap is %lld", n, (long long)cap);
    if (n == 0) return CDFCI_OK;
    unsigned long long *dk = nullptr;
    double *dc = nullptr, *db = nullptr;
    if (cudaMalloc(&dk, (size_t)n * 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&dc, (size_t)n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&db, (size_t)n * sizeof(double)) != cudaSuccess) {
        cudaFree(dk); cudaFree(dc); cudaFree(db);
        return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    }
    cudaError_t e = cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = launch_export(c->P, c->d_st, dk, dc, db, n, c->d_counter, c->stream);
    if (e == cudaSuccess && keys) e = cudaMemcpyAsync(keys, dk, (size_t)n * 2 * sizeof(uint64_t), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && cv) e = cudaMemcpyAsync(cv, dc, (size_t)n * sizeof(double), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && bv) e = cudaMemcpyAsync(bv, db, (size_t)n * sizeof(double), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(dk); cudaFree(dc); cudaFree(db);
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "export: %s", cudaGetErrorString(e));
    return CDFCI_OK;
}

CDFCI_API int cdfci_set_initial(cdfci_handle c, const uint64_t *keys, const double *cv, int64_t n) {
    if (!c || !keys || !cv) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "start vectors are for one state (num_states = 1)");
    if (n < 1) return fail(CDFCI_ERR_ARG, "n = %lld, need at least one entry", (long long)n);
    if (n > c->P.max_entries) return fail(CDFCI_ERR_TABLE_FULL, "%lld entries exceed max_load of the table", (long long)n);
    std::vector<uint64_t> hk;
    std::vector<double> hc;
    int rc = copy_in(hk, keys, (size_t)n * 2);
    if (!rc) rc = copy_in(hc, cv, (size_t)n);
    if (!rc) rc = check_keys(c, hk, n);
    if (rc) return rc;
    bool any = false;
    for (double x : hc) {
        if (!std::isfinite(x)) return fail(CDFCI_ERR_ARG, "non-finite start coefficient");
        any = any || x != 0.0;
    }
    if (!any) return fail(CDFCI_ERR_ARG, "every start coefficient is zero");
    CK(cudaStreamSynchronize(c->stream));
    DevTemp tmp;
    unsigned long long *dk = tmp.put(std::vector<unsigned long long>(hk.begin(), hk.end()), c->stream);
    double *dc = tmp.put(hc, c->stream);
    if (!dk || !dc) return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    rc = reset_state(c);
    if (rc) return rc;
    if (!c->block) {
        CK(launch_init_state(c->d_st, c->d_rec, hk[0], hk[1], hc[0], c->stream));
        rc = run_iterations(c, 1);
        for (int64_t k = 1; !rc && k < n; ++k) {
            CK(launch_force_next(c->d_rec, dk, dc, k, c->stream));
            rc = run_iterations(c, 1);
        }
        if (rc) return rc;
    } else {
        // the candidates of every start column: at most n columns' elements and the n entries
        const long long nh_eff = c->P.doubles_vanish ? c->P.seg[2] : c->P.seg[5];
        rc = grow_candidates(c, (long long)n * nh_eff + n + 64);
        if (rc) return rc;
        for (int64_t k = 0; k < n; ++k) {
            CK(launch_mc_start(c->P, c->mb, hk[2 * k], hk[2 * k + 1], hc[k], k == 0 ? 1 : 0, c->stream));
            CK(launch_mc_scatter_finalize(c->P, c->mb, c->stream));
        }
    }
    CK(cudaStreamSynchronize(c->stream));
    return fill_stats(c, nullptr);
}

CDFCI_API int cdfci_checkpoint(cdfci_handle c, cdfci_checkpoint_header *hdr, uint64_t *keys, double *cv, double *bv,
                               uint8_t *flags, int64_t cap) {
    if (!c || !hdr) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "checkpoints are for one state (num_states = 1)");
    int rc = fill_stats(c, nullptr);                   // m = 1: the pending b of the last coordinate is in the table
    if (rc) return rc;
    cdfci_checkpoint_header h;
    memset(&h, 0, sizeof(h));
    h.version = 1;
    h.N = c->N; h.n_alpha = c->na; h.n_beta = c->nb;
    h.num_coordinates = c->block ? c->mb.m : 1;
    h.n_entries = c->h_st->n_slots;
    if (!c->block) {
        CdRecord R;
        CdPartial F;
        DevTemp tmp;
        CdPartial *dF = tmp.alloc<CdPartial>(1);
        if (!dF) return fail(CDFCI_ERR_NOMEM, "device allocation failed");
        CK(launch_ckpt_fold(c->d_part, c->grid, dF, c->stream));
        CK(cudaMemcpyAsync(&F, dF, sizeof(F), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(&R, c->d_rec, sizeof(R), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (R.forced) return fail(CDFCI_ERR_ARG, "a start step is pending (run cdfci_step first)");
        h.have_prev = R.have_prev; h.done = R.done;
        h.mu[0] = R.mu.hi; h.mu[1] = R.mu.lo; h.alpha[0] = R.alpha.hi; h.alpha[1] = R.alpha.lo;
        h.scale[0] = 1.0; h.scale[1] = 0.0;
        h.dx = R.dx; h.energy = R.energy; h.last_gamma = 0.0;
        h.iterations = R.iterations; h.nnz_c = R.nnz_c; h.n_slots = R.n_slots; h.elements = R.elements;
        h.applied = R.applied; h.dropped = R.dropped; h.inserted = R.inserted; h.last_column = R.last_column;
        h.prev_key[0] = R.a; h.prev_key[1] = R.b;
        h.prev_c = R.c_new; h.prev_Hii = R.Hii; h.prev_eta = R.eta; h.prev_mu_g = R.mu_g;
        h.has_best = R.have_prev && F.slot >= 0 ? 1 : 0;
        h.best_key[0] = F.ka; h.best_key[1] = F.kb; h.best_gbits = F.gbits;
        h.best_b = F.bj; h.best_c = F.cj; h.gather = R.have_prev ? F.gather : 0.0;
        h.pending[0] = R.have_prev ? F.elements : 0; h.pending[1] = R.have_prev ? F.applied : 0;
        h.pending[2] = R.have_prev ? F.dropped : 0; h.pending[3] = R.have_prev ? F.inserted : 0;
        h.pending_err = R.have_prev ? F.err : 0;
    } else {
        McState ms;
        CK(cudaMemcpyAsync(&ms, c->mb.ms, sizeof(ms), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        h.done = ms.done;
        h.mu[0] = ms.mu.hi; h.mu[1] = ms.mu.lo; h.alpha[0] = ms.alpha.hi; h.alpha[1] = ms.alpha.lo;
        h.scale[0] = ms.scale.hi; h.scale[1] = ms.scale.lo;
        h.dx = ms.dx; h.energy = ms.energy; h.last_gamma = ms.last_gamma;
        h.iterations = ms.iterations; h.nnz_c = ms.nnz_c; h.n_slots = ms.n_slots; h.elements = ms.elements;
        h.applied = ms.applied; h.dropped = ms.dropped; h.inserted = ms.inserted; h.last_column = ms.last_column;
        h.reduced_iterations = ms.eig_iters_total;
    }
    *hdr = h;
    const long long n = h.n_entries;
    if (cap < n) return fail(CDFCI_ERR_CAPACITY, "%lld entries stored, cap is %lld", n, (long long)cap);
    if (!keys || !cv || !bv) return fail(CDFCI_ERR_ARG, "NULL row array");
    DevTemp tmp;
    unsigned long long *dk = tmp.alloc<unsigned long long>((size_t)n * 2);
    double *dc = tmp.alloc<double>((size_t)n), *db = tmp.alloc<double>((size_t)n);
    unsigned char *df = tmp.alloc<unsigned char>((size_t)n);
    if (!dk || !dc || !db || !df) return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    CK(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned long long), c->stream));
    CK(launch_ckpt_export(c->P, dk, dc, db, df, n, c->d_counter, c->stream));
    CK(cudaMemcpyAsync(keys, dk, (size_t)n * 2 * sizeof(uint64_t), cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(cv, dc, (size_t)n * sizeof(double), cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(bv, db, (size_t)n * sizeof(double), cudaMemcpyDefault, c->stream));
    if (flags) CK(cudaMemcpyAsync(flags, df, (size_t)n, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return CDFCI_OK;
}

CDFCI_API int cdfci_restore(cdfci_handle c, const cdfci_checkpoint_header *hdr, const uint64_t *keys, const double *cv,
                            const double *bv, const uint8_t *flags) {
    if (!c || !hdr || !keys || !cv || !bv) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "checkpoints are for one state (num_states = 1)");
    const cdfci_checkpoint_header h = *hdr;
    if (h.version != 1) return fail(CDFCI_ERR_ARG, "checkpoint version %d, expected 1", h.version);
    if (h.N != c->N || h.n_alpha != c->na || h.n_beta != c->nb)
        return fail(CDFCI_ERR_ARG, "checkpoint of N = %d, %d + %d electrons; handle has N = %d, %d + %d", h.N, h.n_alpha,
                    h.n_beta, c->N, c->na, c->nb);
    if ((h.num_coordinates > 1) != c->block)
        return fail(CDFCI_ERR_ARG, "checkpoint of m = %d cannot resume on a handle with m %s", h.num_coordinates,
                    c->block ? "> 1" : "= 1");
    const long long n = h.n_entries;
    if (n < 1) return fail(CDFCI_ERR_ARG, "checkpoint with %lld entries", n);
    if (n > c->P.max_entries) return fail(CDFCI_ERR_TABLE_FULL, "%lld entries exceed max_load of the table", n);
    std::vector<uint64_t> hk;
    std::vector<double> hc, hb;
    std::vector<uint8_t> hf;
    int rc = copy_in(hk, keys, (size_t)n * 2);
    if (!rc) rc = copy_in(hc, cv, (size_t)n);
    if (!rc) rc = copy_in(hb, bv, (size_t)n);
    if (!rc && flags) rc = copy_in(hf, flags, (size_t)n);
    if (!rc) rc = check_keys(c, hk, n);
    if (rc) return rc;
    if (c->block) {
        long long nc = 0;
        for (uint8_t f : hf) nc += f & 1;
        // a checkpoint written after a long start vector may list more candidates than one iteration makes
        rc = grow_candidates(c, nc + c->mb.m + 64);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(c->stream));
    DevTemp tmp;
    unsigned long long *dk = tmp.put(std::vector<unsigned long long>(hk.begin(), hk.end()), c->stream);
    double *dc = tmp.put(hc, c->stream), *db = tmp.put(hb, c->stream);
    unsigned char *df = hf.empty() ? nullptr : tmp.put(std::vector<unsigned char>(hf.begin(), hf.end()), c->stream);
    if (!dk || !dc || !db || (!hf.empty() && !df)) return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    rc = reset_state(c);
    if (rc) return rc;
    if (!c->block) {
        CK(launch_ckpt_import(c->P, c->d_st, dk, dc, db, nullptr, n, nullptr, nullptr, 0, c->stream));
        CdRecord R;
        memset(&R, 0, sizeof(R));
        R.a = h.prev_key[0]; R.b = h.prev_key[1]; R.slot = 0;
        R.c_new = h.prev_c; R.Hii = h.prev_Hii; R.eta = h.prev_eta; R.mu_g = h.prev_mu_g;
        R.mu = dd{h.mu[0], h.mu[1]}; R.alpha = dd{h.alpha[0], h.alpha[1]};
        R.dx = h.dx; R.energy = h.energy;
        R.iterations = h.iterations; R.nnz_c = h.nnz_c; R.n_slots = h.n_slots; R.elements = h.elements;
        R.applied = h.applied; R.dropped = h.dropped; R.inserted = h.inserted; R.last_column = h.last_column;
        R.forced = 0; R.have_prev = h.have_prev ? 1 : 0; R.done = h.done;
        CdPartial F;
        memset(&F, 0, sizeof(F));
        F.gather = h.gather; F.gbits = h.has_best ? h.best_gbits : 0ull;
        F.ka = h.has_best ? h.best_key[0] : ~0ull; F.kb = h.has_best ? h.best_key[1] : ~0ull;
        F.slot = h.has_best ? 0 : -1;
        F.bj = h.best_b; F.cj = h.best_c;
        F.elements = (int)h.pending[0]; F.applied = (int)h.pending[1]; F.dropped = (int)h.pending[2];
        F.inserted = (int)h.pending[3]; F.err = h.pending_err;
        CK(launch_ckpt_restore_m1(c->P, c->d_st, c->d_rec, c->d_part, c->grid, R, F, c->stream));
    } else {
        McState ms;
        memset(&ms, 0, sizeof(ms));
        ms.mu = dd{h.mu[0], h.mu[1]}; ms.alpha = dd{h.alpha[0], h.alpha[1]}; ms.scale = dd{h.scale[0], h.scale[1]};
        ms.dx = h.dx; ms.energy = h.energy; ms.last_gamma = h.last_gamma;
        ms.iterations = h.iterations; ms.nnz_c = h.nnz_c; ms.n_slots = h.n_slots; ms.elements = h.elements;
        ms.applied = h.applied; ms.dropped = h.dropped; ms.inserted = h.inserted; ms.last_column = h.last_column;
        ms.done = h.done; ms.eig_iters_total = h.reduced_iterations;
        CK(cudaMemcpyAsync(c->mb.ms, &ms, sizeof(ms), cudaMemcpyHostToDevice, c->stream));
        IterState t;
        memset(&t, 0, sizeof(t));
        t.scale = ms.scale;
        t.iterations = ms.iterations; t.nnz_c = ms.nnz_c; t.n_slots = ms.n_slots; t.elements = ms.elements;
        t.applied = ms.applied; t.dropped = ms.dropped; t.inserted = ms.inserted; t.last_column = ms.last_column;
        t.mu = ms.mu; t.alpha = ms.alpha; t.dx = ms.dx; t.energy = ms.energy; t.eig_iters = ms.eig_iters_total;
        t.done = ms.done;
        CK(cudaMemcpyAsync(c->d_st, &t, sizeof(t), cudaMemcpyHostToDevice, c->stream));
        CK(launch_ckpt_import(c->P, c->d_st, dk, dc, db, df, n, c->mb.cand, &c->mb.ms->n_cand, c->mb.cap_cand,
                              c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return fill_stats(c, nullptr);
}

namespace {
// RDMs into device buffers owned by the caller of this helper (N*N and N^4)
int rdm_device(cdfci_ctx *c, double *g1, double *g2) {
    const size_t n2 = (size_t)c->P.N * c->P.N, n4 = n2 * n2;
    double *raw1 = nullptr, *raw2 = nullptr, *nrm = nullptr;
    if (cudaMalloc(&raw1, n2 * sizeof(double)) != cudaSuccess || cudaMalloc(&raw2, n4 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&nrm, sizeof(double)) != cudaSuccess) {
        cudaFree(raw1); cudaFree(raw2); cudaFree(nrm);
        return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    }
    cudaError_t e = launch_rdm(c->P, c->d_st, raw1, raw2, nrm, g1, g2, c->stream);
    double norm = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&norm, nrm, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(raw1); cudaFree(raw2); cudaFree(nrm);
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "rdm: %s", cudaGetErrorString(e));
    if (!(norm > 0.0)) return fail(CDFCI_ERR_ARG, "rdm: the stored vector is zero");
    return CDFCI_OK;
}
}  // namespace

CDFCI_API int cdfci_rdm(cdfci_handle c, double *rdm1, double *rdm2) {
    if (!c || !rdm1) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "RDMs are for one state (num_states = 1)");
    int rc = fill_stats(c, nullptr);
    if (rc) return rc;
    const size_t n2 = (size_t)c->P.N * c->P.N, n4 = n2 * n2;
    double *g1 = nullptr, *g2 = nullptr;
    if (cudaMalloc(&g1, n2 * sizeof(double)) != cudaSuccess || cudaMalloc(&g2, n4 * sizeof(double)) != cudaSuccess) {
        cudaFree(g1); cudaFree(g2);
        return fail(CDFCI_ERR_NOMEM, "device allocation failed");
    }
    rc = rdm_device(c, g1, g2);
    cudaError_t e = cudaSuccess;
    if (!rc) e = cudaMemcpyAsync(rdm1, g1, n2 * sizeof(double), cudaMemcpyDefault, c->stream);
    if (!rc && e == cudaSuccess && rdm2) e = cudaMemcpyAsync(rdm2, g2, n4 * sizeof(double), cudaMemcpyDefault, c->stream);
    if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(g1); cudaFree(g2);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "rdm copy: %s", cudaGetErrorString(e));
    return CDFCI_OK;
}

CDFCI_API int cdfci_gradient(cdfci_handle c, double *dE_dh, double *dE_dg, double *dE_dkappa) {
    if (!c) return fail(CDFCI_ERR_ARG, "NULL argument");
    if (c->xcd) return fail(CDFCI_ERR_UNIMPLEMENTED, "gradients are for one state (num_states = 1)");
    int rc = fill_stats(c, nullptr);
    if (rc) return rc;
    const int N = c->P.N;
    const size_t n2 = (size_t)N * N, n4 = n2 * n2;
    double *g1 = nullptr, *g2 = nullptr, *F = nullptr, *oh = nullptr, *og = nullptr, *ok = nullptr;
    bool okm = cudaMalloc(&g1, n2 * sizeof(double)) == cudaSuccess && cudaMalloc(&g2, n4 * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&F, n2 * sizeof(double)) == cudaSuccess && cudaMalloc(&oh, n2 * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&og, n4 * sizeof(double)) == cudaSuccess && cudaMalloc(&ok, n2 * sizeof(double)) == cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!okm) rc = fail(CDFCI_ERR_NOMEM, "device allocation failed");
    if (!rc) rc = rdm_device(c, g1, g2);
    if (!rc) e = launch_gradient(N, c->d_h, c->d_g, g1, g2, F, dE_dh ? oh : nullptr, dE_dg ? og : nullptr,
                                 dE_dkappa ? ok : nullptr, c->stream);
    if (!rc && e == cudaSuccess && dE_dh) e = cudaMemcpyAsync(dE_dh, oh, n2 * sizeof(double), cudaMemcpyDefault, c->stream);
    if (!rc && e == cudaSuccess && dE_dg) e = cudaMemcpyAsync(dE_dg, og, n4 * sizeof(double), cudaMemcpyDefault, c->stream);
    if (!rc && e == cudaSuccess && dE_dkappa) e = cudaMemcpyAsync(dE_dkappa, ok, n2 * sizeof(double), cudaMemcpyDefault, c->stream);
    if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(g1); cudaFree(g2); cudaFree(F); cudaFree(oh); cudaFree(og); cudaFree(ok);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "gradient: %s", cudaGetErrorString(e));
    return CDFCI_OK;
}

// ---------------------------------------------------------------------------
// Batches of independent m = 1 solvers
// ---------------------------------------------------------------------------
}  // extern "C"

struct cdfci_batch {
    std::vector<cdfci_ctx *> hs;       // every handle, in the caller's order
    std::vector<cdfci_ctx *> one;      // m = 1 handles: one persistent launch, a cluster per problem
    std::vector<int> one_at;           // their positions in hs
    std::vector<cdfci_ctx *> blk;      // m > 1 handles: one graph branch each
    std::vector<int> blk_at;
    CdInstance *d_inst = nullptr;
    int cluster = 1;
    size_t smem = 0;
    cudaStream_t stream = nullptr;     // the batch's stream (handle 0's)
    long long chunk = 1 << 16;
    cudaGraphExec_t graph = nullptr;   // the m = 1 group's launch of graph_iters iterations
    long long graph_iters = 0;
    std::vector<cudaStream_t> br;      // the m > 1 group: a branch stream per handle ...
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t mgraph = nullptr;  // ... and one graph of mchunk iterations of every branch
    int mchunk = 8;
};

namespace {
int batch_graph(cdfci_batch *b, long long k) {
    if (b->graph && b->graph_iters == k) return CDFCI_OK;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_cd_loop_batch(b->d_inst, (int)b->one.size(), b->cluster, b->smem, k, b->stream);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(CDFCI_ERR_CUDA, "capture of the batched launch failed");
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    b->graph_iters = k;
    return CDFCI_OK;
}

// The m > 1 group: one graph in which every handle's mchunk iterations (its own
// kernels and launch shapes) form a branch of their own, forked from the batch
// stream and joined back, so that the problems' iterations run side by side.
int batch_mgraph(cdfci_batch *b) {
    if (b->mgraph) { cudaGraphExecDestroy(b->mgraph); b->mgraph = nullptr; }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    for (size_t i = 0; i < b->blk.size() && e == cudaSuccess; ++i) {
        cdfci_ctx *c = b->blk[i];
        e = cudaStreamWaitEvent(b->br[i], b->fork, 0);
        for (int it = 0; it < b->mchunk && e == cudaSuccess; ++it) e = launch_mc_iteration(c->P, c->mb, b->br[i]);
        if (e == cudaSuccess) e = cudaEventRecord(b->join[i], b->br[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(CDFCI_ERR_CUDA, "capture of the batched multicoordinate iteration failed");
    }
    e = cudaGraphInstantiate(&b->mgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(CDFCI_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return CDFCI_OK;
}

void batch_free(cdfci_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->mgraph) cudaGraphExecDestroy(b->mgraph);
    for (cudaStream_t s : b->br) if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->d_inst);
    delete b;
}
}  // namespace

extern "C" {

CDFCI_API int cdfci_batch_create(const cdfci_handle *hs, int n, cdfci_batch_handle *out) {
    if (!out) return fail(CDFCI_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (!hs || n < 1) return fail(CDFCI_ERR_ARG, "empty batch");
    int first_one = -1;
    for (int k = 0; k < n; ++k) {
        if (!hs[k]) return fail(CDFCI_ERR_ARG, "handle %d is NULL", k);
        if (hs[k]->xcd) return fail(CDFCI_ERR_ARG, "handle %d has num_states > 1 (batches take one-state solvers)", k);
        for (int q = 0; q < k; ++q)
            if (hs[q] == hs[k]) return fail(CDFCI_ERR_ARG, "handle %d appears twice", k);
        if (hs[k]->block) continue;
        if (hs[k]->gridmode)
            return fail(CDFCI_ERR_ARG, "handle %d runs on %d CTAs, more than a cluster (batches take grid_blocks <= 16)",
                        k, hs[k]->grid);
        if (first_one < 0) first_one = k;
        if (hs[k]->grid != hs[first_one]->grid)
            return fail(CDFCI_ERR_ARG, "handle %d uses %d CTAs per problem, handle %d uses %d (create the m = 1 "
                        "solvers with the same grid_blocks)", k, hs[k]->grid, first_one, hs[first_one]->grid);
    }
    cdfci_batch *b = new (std::nothrow) cdfci_batch;
    if (!b) return fail(CDFCI_ERR_NOMEM, "host allocation failed");
    b->hs.assign(hs, hs + n);
    for (int k = 0; k < n; ++k) {
        if (hs[k]->block) { b->blk.push_back(hs[k]); b->blk_at.push_back(k); }
        else { b->one.push_back(hs[k]); b->one_at.push_back(k); }
    }
    b->stream = hs[0]->stream;
    // every handle's queued work is complete before the batch touches its state
    for (int k = 0; k < n; ++k)
        if (cudaStreamSynchronize(hs[k]->stream) != cudaSuccess) { batch_free(b); return fail(CDFCI_ERR_CUDA, "stream sync failed"); }
    if (!b->one.empty()) {
        b->cluster = b->one[0]->grid;
        b->chunk = b->one[0]->chunk;
        std::vector<CdInstance> inst(b->one.size());
        for (size_t k = 0; k < b->one.size(); ++k) {
            cdfci_ctx *c = b->one[k];
            inst[k] = CdInstance{c->P, c->d_st, c->d_rec, c->d_part};
            b->smem = std::max(b->smem, cd_dynamic_smem(c->P));
        }
        if (cudaMalloc(&b->d_inst, inst.size() * sizeof(CdInstance)) != cudaSuccess) {
            batch_free(b);
            return fail(CDFCI_ERR_NOMEM, "device allocation failed");
        }
        if (cudaMemcpy(b->d_inst, inst.data(), inst.size() * sizeof(CdInstance), cudaMemcpyHostToDevice) != cudaSuccess) {
            batch_free(b);
            return fail(CDFCI_ERR_CUDA, "copy of the instance table failed");
        }
    }
    if (!b->blk.empty()) {
        b->mchunk = b->blk[0]->mchunk;
        b->br.assign(b->blk.size(), nullptr);
        b->join.assign(b->blk.size(), nullptr);
        bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
        for (size_t i = 0; i < b->blk.size() && ok; ++i)
            ok = cudaStreamCreateWithFlags(&b->br[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) { batch_free(b); return fail(CDFCI_ERR_CUDA, "stream or event creation failed"); }
        const int rc = batch_mgraph(b);
        if (rc) { batch_free(b); return rc; }
    }
    *out = b;
    return CDFCI_OK;
}

CDFCI_API int cdfci_batch_step(cdfci_batch_handle b, int64_t n_iter, cdfci_stats *stats) {
    if (!b) return fail(CDFCI_ERR_ARG, "NULL batch");
    if (n_iter < 0) return fail(CDFCI_ERR_ARG, "n_iter < 0");
    // work a handle queued on its own stream (a solo step) completes first
    for (cdfci_ctx *c : b->hs)
        if (c->stream != b->stream) CK(cudaStreamSynchronize(c->stream));
    // m = 1 group: the persistent batch launch
    long long left = b->one.empty() ? 0 : n_iter;
    while (left > 0) {
        const long long k = std::min(left, b->chunk);
        int rc = batch_graph(b, k);
        if (rc) return rc;
        CK(cudaGraphLaunch(b->graph, b->stream));
        left -= k;
    }
    if (!b->one.empty()) CK(launch_cd_finalize_batch(b->d_inst, (int)b->one.size(), b->cluster, b->stream));
    // m > 1 group: graphs of mchunk iterations of every problem side by side, then the rest
    if (!b->blk.empty()) {
        for (int64_t i = 0; i < n_iter / b->mchunk; ++i) {
            bool rebuild = false;
            for (cdfci_ctx *c : b->blk) {
                if (!c->prm.z_threshold_search) continue;
                CK(cudaStreamSynchronize(b->stream));
                bool changed = false;
                const int rc = maybe_raise_tau(c, &changed);      // tau is a launch parameter of the graph
                if (rc) return rc;
                rebuild = rebuild || changed;
            }
            if (rebuild) {
                const int rc = batch_mgraph(b);
                if (rc) return rc;
            }
            CK(cudaGraphLaunch(b->mgraph, b->stream));
        }
        for (cdfci_ctx *c : b->blk)
            for (int64_t r = 0; r < n_iter % b->mchunk; ++r) CK(launch_mc_iteration(c->P, c->mb, b->stream));
    }
    for (size_t k = 0; k < b->one.size(); ++k)
        CK(cudaMemcpyAsync(b->one[k]->h_st, b->one[k]->d_st, sizeof(IterState), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    int first = CDFCI_OK;
    for (size_t k = 0; k < b->one.size(); ++k) {
        const int rc = stats_from_snapshot(b->one[k], stats ? stats + b->one_at[k] : nullptr);
        if (rc && !first) first = rc;
    }
    for (size_t k = 0; k < b->blk.size(); ++k) {
        const int rc = fill_stats(b->blk[k], stats ? stats + b->blk_at[k] : nullptr);
        if (rc && !first) first = rc;
    }
    return first;
}

CDFCI_API void cdfci_batch_destroy(cdfci_batch_handle b) {
    if (!b) return;
    batch_free(b);
}

CDFCI_API int cdfci_autotune(const double *h, const double *g, int N, int n_alpha, int n_beta, cdfci_params *params,
                             double seconds, cdfci_tune_report *report) {
    if (!params) return fail(CDFCI_ERR_ARG, "NULL params");
    if (!(seconds > 0.0)) return fail(CDFCI_ERR_ARG, "seconds must be > 0");
    if (params->num_states > 1) return fail(CDFCI_ERR_ARG, "the autotuner picks m for one state (num_states = 1)");
    struct Cand { int m, grid; };
    std::vector<Cand> cs;
    cs.push_back({1, params->grid_blocks});
    for (int gb : {1, 2, 4, 8, 16, 32, 64, 128})
        if (gb != params->grid_blocks) cs.push_back({1, gb});
    for (int m : {4, 16, 64, 256})
        if (m <= mc_max_m()) cs.push_back({m, params->grid_blocks});
    cdfci_tune_report rep;
    memset(&rep, 0, sizeof(rep));
    const double share = seconds / (double)cs.size();
    double target = 0.0, best = 1e300;
    for (size_t k = 0; k < cs.size() && k < 16; ++k) {
        cdfci_params p = *params;
        p.num_coordinates = cs[k].m;
        p.grid_blocks = cs[k].grid;
        cdfci_handle hd = nullptr;
        int rc = cdfci_create(h, g, N, n_alpha, n_beta, &p, &hd);
        if (rc) return rc;
        const int resolved_grid = cs[k].m == 1 ? hd->grid : 0;
        cdfci_stats st0, st;
        rc = cdfci_get_stats(hd, &st0);
        st = st0;
        double spent = 0.0, reached = -1.0;
        long long it = 0;
        const int64_t chunk = cs[k].m == 1 ? 256 : 4;
        // the first candidate runs its share and sets the target energy; the others run until they reach it
        const double limit = k == 0 ? share : 2.0 * share;
        while (!rc && spent < limit && !st.converged) {
            const auto t0 = std::chrono::steady_clock::now();
            rc = cdfci_step(hd, chunk, &st);
            spent += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (!rc) it += chunk;
            if (!rc && k > 0 && st.energy <= target) { reached = spent; break; }
        }
        if (rc == CDFCI_ERR_TABLE_FULL) rc = CDFCI_OK;  // scored by what it reached
        cdfci_destroy(hd);
        if (rc) return rc;
        if (k == 0) { target = st.energy; reached = spent; }
        rep.m[k] = cs[k].m;
        rep.grid_blocks[k] = resolved_grid;
        rep.iterations[k] = it;
        rep.seconds[k] = spent;
        rep.energy_drop[k] = st0.energy - st.energy;
        rep.score[k] = reached;                      // seconds to the target energy, -1 if not reached
        if (reached >= 0.0 && reached < best) { best = reached; rep.chosen = (int)k; }
        rep.n = (int)k + 1;
    }
    params->num_coordinates = rep.m[rep.chosen];
    if (rep.m[rep.chosen] == 1) params->grid_blocks = rep.grid_blocks[rep.chosen];
    if (report) *report = rep;
    return CDFCI_OK;
}

CDFCI_API int cdfci_last_step(cdfci_handle c, uint64_t *keys, double *eta, int64_t cap, int64_t *m_out) {
    if (!c || !m_out) return fail(CDFCI_ERR_ARG, "NULL argument");
    int rc = fill_stats(c, nullptr);
    if (rc) return rc;
    if (c->xcd) {
        XState x;
        CK(cudaMemcpy(&x, c->xb.xs, sizeof(x), cudaMemcpyDeviceToHost));
        *m_out = 1;
        if (cap < 1) return fail(CDFCI_ERR_CAPACITY, "cap < 1");
        uint64_t k[2] = {x.A, x.B};
        if (keys) CK(cudaMemcpy(keys, k, sizeof(k), cudaMemcpyDefault));
        if (eta) CK(cudaMemcpy(eta, &x.eta, sizeof(double), cudaMemcpyDefault));
        return CDFCI_OK;
    }
    if (c->block) {
        McState ms;
        CK(cudaMemcpy(&ms, c->mb.ms, sizeof(ms), cudaMemcpyDeviceToHost));
        const int m = ms.m_sel;
        *m_out = m;
        if (cap < m) return fail(CDFCI_ERR_CAPACITY, "%d coordinates, cap is %lld", m, (long long)cap);
        std::vector<McSel> sel(m > 0 ? m : 1);
        std::vector<double> et(m > 0 ? m : 1);
        if (m > 0) {
            CK(cudaMemcpy(sel.data(), c->mb.sel, m * sizeof(McSel), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(et.data(), c->mb.eta, m * sizeof(double), cudaMemcpyDeviceToHost));
        }
        std::vector<uint64_t> kk(2 * (m > 0 ? m : 1));
        for (int i = 0; i < m; ++i) { kk[2 * i] = sel[i].A; kk[2 * i + 1] = sel[i].B; }
        if (keys && m > 0) CK(cudaMemcpy(keys, kk.data(), 2 * m * sizeof(uint64_t), cudaMemcpyDefault));
        if (eta && m > 0) CK(cudaMemcpy(eta, et.data(), m * sizeof(double), cudaMemcpyDefault));
        return CDFCI_OK;
    }
    *m_out = 1;
    if (cap < 1) return fail(CDFCI_ERR_CAPACITY, "cap < 1");
    uint64_t k[2] = {c->h_st->last_a, c->h_st->last_b};
    double e = c->h_st->last_eta;
    if (keys) CK(cudaMemcpy(keys, k, sizeof(k), cudaMemcpyDefault));
    if (eta) CK(cudaMemcpy(eta, &e, sizeof(e), cudaMemcpyDefault));
    return CDFCI_OK;
}

CDFCI_API void cdfci_destroy(cdfci_handle c) { free_ctx(c); }

}  // extern "C"
