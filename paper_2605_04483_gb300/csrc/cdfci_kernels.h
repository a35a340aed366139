// Host-side launch wrappers of the kernels in cdfci_kernels.cu (library-internal).
#pragma once
#include <cuda_runtime.h>

#include "cdfci_internal.cuh"

namespace cdfci {

cudaError_t launch_cd_loop(const Problem &P, IterState *st, CdRecord *rec, CdPartial *part, int cluster,
                           long long n_iter, cudaStream_t s);
size_t cd_dynamic_smem(const Problem &P);
int cd_pick_cluster(int want, size_t smem);
cudaError_t launch_cd_finalize(const Problem &P, IterState *st, CdRecord *rec, CdPartial *part, int cluster,
                               cudaStream_t s);
cudaError_t launch_column(const Problem &P, unsigned long long A, unsigned long long B, unsigned long long *keys,
                          double *vals, long long cap, unsigned long long *counter, cudaStream_t s);
cudaError_t launch_export(const Problem &P, const IterState *st, unsigned long long *keys, double *c, double *b,
                          long long cap, unsigned long long *counter, cudaStream_t s);
cudaError_t launch_rq(const Problem &P, IterState *st, long long *list, long long cap, unsigned long long *counter,
                      double *partial, int nblocks, double *out, cudaStream_t s);
cudaError_t launch_setup(double *h, double *g, int N, double *J, double *K, double *W3, double *V3, int *status,
                         int *has_doubles, int sym4, cudaStream_t s);
cudaError_t launch_init_state(IterState *st, CdRecord *rec, unsigned long long A, unsigned long long B, double eta,
                              cudaStream_t s);
cudaError_t launch_force_next(CdRecord *rec, const unsigned long long *keys, const double *c, long long k,
                              cudaStream_t s);
// xCDFCI (Algorithm 3): k1 = K + 1 states
struct XBuffers {
    XState *xs;
    IterState *st;
    double *rows;                  // capacity x 2 k1: C row, B row
    long long *cand;               // candidate slots (deduplicated by the mark)
    long long cap_cand;
    double *gathp;                 // per scatter block: k1 gather sums
    void *bbest;                   // per select block: its best candidate
    unsigned int *counter;         // last-block counter of the selection
    int nscatter, nselect;
};
int x_scatter_blocks();
size_t x_block_bytes();
cudaError_t launch_x_start(const Problem &P, const XBuffers &b, unsigned long long A, unsigned long long B, int k,
                           cudaStream_t s);
cudaError_t launch_x_iteration(const Problem &P, const XBuffers &b, cudaStream_t s);
cudaError_t launch_x_energies(const XBuffers &b, cudaStream_t s);
cudaError_t launch_x_export(const Problem &P, const XBuffers &b, int k1, unsigned long long *keys, double *C,
                            double *B, long long cap, unsigned long long *counter, cudaStream_t s);
cudaError_t launch_x_diag_list(const Problem &P, const unsigned long long *keys, long long n, double *out,
                               cudaStream_t s);

// OptOrbFCI (Algorithm 4): orbital subproblem kernels
cudaError_t oo_contract(const double *in, const double *U, double *out, long long A, int M, int N, long long B,
                        cudaStream_t s);
cudaError_t oo_grad(const double *hU, const double *g1, const double *g3, const double *g2, double *G, int M, int N,
                    cudaStream_t s);
cudaError_t oo_dot(const double *x, const double *y, long long n, double *out, cudaStream_t s);
cudaError_t oo_axpy(const double *x, const double *z, double t, double *y, long long n, cudaStream_t s);
cudaError_t oo_scale(double *x, const double *sq, long long n, cudaStream_t s);
cudaError_t oo_gram(const double *X, double *Gm, int M, int N, cudaStream_t s);
cudaError_t oo_ns(const double *X, const double *Gm, double *Xn, int M, int N, cudaStream_t s);

// checkpoint / restore
cudaError_t launch_ckpt_export(const Problem &P, unsigned long long *keys, double *c, double *b, unsigned char *flags,
                               long long cap, unsigned long long *counter, cudaStream_t s);
cudaError_t launch_ckpt_fold(const CdPartial *gpart, int G, CdPartial *out, cudaStream_t s);
cudaError_t launch_ckpt_import(const Problem &P, IterState *st, const unsigned long long *keys, const double *c,
                               const double *b, const unsigned char *flags, long long n, long long *cand, int *n_cand,
                               long long cap_cand, cudaStream_t s);
cudaError_t launch_ckpt_restore_m1(const Problem &P, IterState *st, CdRecord *rec, CdPartial *gpart, int G,
                                   const CdRecord &r, const CdPartial &folded, cudaStream_t s);

// Device buffers of the multicoordinate iteration.
// One column's single excitations in global memory (built once per iteration for the
// scatter): alpha entries [0, nsA), beta entries [nsA, nsA + nsB).
struct __align__(16) ColEnt {
    unsigned long long key, h;     // the changed string and its hash (hash_alpha / hash_beta)
    int goff;                      // alpha: (i N + a) N^2; beta: j N + b
    int info;                      // sign | i << 8 | a << 16 | momentum transfer << 24
    int pad0, pad1;
};
// The scatter's work items per column: opposite-spin (ab), same-spin (aa, bb) and singles (s)
// items; *_ch = chunks of the looped factor per lane group of 32.
struct McGeom {
    int nsA, nsB;
    int n_ab, ab_ch, n_aa, aa_ch, n_bb, bb_ch, n_s;
    int per_col;
};
struct McBuffers {
    McState *ms;
    IterState *st;
    long long *cand;               // candidate slots (deduplicated)
    unsigned long long *gkey;      // their choice keys
    unsigned int *hist;            // 4096-bin radix histogram, then the last-block counter
    McSel *sel, *inbin, *ties;     // chosen set, threshold-digit candidates, exact-tie scratch
    double *cI, *bI, *Hdiag, *HIIc, *w, *thr, *eta, *gathp;   // gathp: m x geom.per_col item partials
    float4 *rowf;                  // per chosen row: (c, b), (H_II c_I, b - H_II c_I) as float-float pairs
    ColEnt *coltab;                // m columns x (nsA + nsB) single excitations
    ColLists *collists;            // m columns' orbital lists
    unsigned int *work;            // the scatter's item counter (reset by k_mc_finalize)
    McGeom geom;
    float *Rh, *Rl;                // reduced matrix R as float-float pairs, leading dimension ldr
    int ldr;
    int m, cand_grid, scatter_grid;
    long long cap_cand;            // entries of cand / gkey / ties
};
size_t mc_eigen_smem(int m);
int mc_ldr(int m);                  // row stride of R for a block of m coordinates
int mc_max_m();
int mc_scatter_grid(const Problem &P);
McGeom mc_geometry(const Problem &P);
cudaError_t mc_configure();
cudaError_t launch_entry(const Problem &P, unsigned long long A1, unsigned long long B1, unsigned long long A2,
                         unsigned long long B2, double *out, cudaStream_t s);
cudaError_t launch_mc_start(const Problem &P, const McBuffers &b, unsigned long long A, unsigned long long B,
                            double eta, int first, cudaStream_t s);
cudaError_t launch_mc_scatter_finalize(const Problem &P, const McBuffers &b, cudaStream_t s);
constexpr int kMcKernels = 8;       // launches of one mCDFCI iteration
cudaError_t launch_mc_iteration(const Problem &P, const McBuffers &b, cudaStream_t s, cudaEvent_t *ev = nullptr);

// the m = 1 loop over more CTAs than a cluster holds (cooperative launch)
cudaError_t launch_cd_loop_grid(const Problem &P, IterState *st, CdRecord *rec, CdPartial *gpart,
                                unsigned long long *xchg, GridRound *rnd, int G, long long n_iter, cudaStream_t s);
int cd_max_grid(size_t smem);

// batches of independent m = 1 problems: one launch, one cluster per instance
cudaError_t launch_cd_loop_batch(const CdInstance *inst, int n_inst, int cluster, size_t smem, long long n_iter,
                                 cudaStream_t s);
cudaError_t launch_cd_finalize_batch(const CdInstance *inst, int n_inst, int cluster, cudaStream_t s);

// reduced density matrices and the energy's derivatives (cdfci_rdm.cu)
cudaError_t launch_rdm(const Problem &P, IterState *st, double *g1_raw, double *g2_raw, double *norm, double *g1,
                       double *g2, cudaStream_t s);
cudaError_t launch_gradient(int N, const double *h, const double *g, const double *G1, const double *G2, double *F,
                            double *dh, double *dg, double *dk, cudaStream_t s);

// sets the message returned by cdfci_last_error() on the calling thread
void set_last_error_message(const char *msg);

}  // namespace cdfci
