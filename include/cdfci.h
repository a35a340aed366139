/*
 * cdfci.h - C-ABI of libcdfci, the GB300 (sm_103a) column-update engine for
 * coordinate-descent FCI (CDFCI, Algorithm 1; mCDFCI, Algorithm 2 of the
 * paper "CDFCI: High-Performance Parallel Software for Quantum Many-Body
 * Eigenvalue Problems").
 *
 * Model.  The Hamiltonian is Eq. (general-ham) over N spatial orbitals with
 * real integrals:
 *   h : N*N doubles, row-major, h[p*N+q] = h_pq (Eq. 1int), symmetric;
 *   g : N^4 doubles, row-major, g[((p*N+q)*N+r)*N+s] = (pq|rs) in chemists'
 *       order, 8-fold symmetric; the physicists' v_pqrs of Eq. (2int) is (pr|qs).
 * A determinant is a key of two 64-bit words {A, B}: bit p of A means spatial
 * orbital p holds an alpha electron, bit p of B a beta electron.  Signs use
 * the Jordan-Wigner order in which every alpha spin-orbital precedes every
 * beta one.  N <= 63 (bit 63 of the beta word marks candidates in the table).
 *
 * Conventions for every call:
 *   - Return value 0 = success, a negative CDFCI_ERR_* code otherwise; the
 *     message of the last failure on the calling thread is cdfci_last_error().
 *   - Pointer arguments may be host or device memory (the library asks the
 *     CUDA driver which); the library copies what it needs and never keeps a
 *     caller pointer.  The caller owns every buffer it passes.
 *   - The library owns all memory behind a handle and frees it in
 *     cdfci_destroy.  No call aborts the process, traps or waits without
 *     bound on the GPU: every device-side loop is bounded and reports
 *     CDFCI_ERR_TABLE_FULL / CDFCI_ERR_TIMEOUT / CDFCI_ERR_NONFINITE instead.
 *   - Energies are Hartree (the unit of h and g), FP64.
 */
#ifndef CDFCI_H
#define CDFCI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CDFCI_OK                 0
#define CDFCI_ERR_ARG           -1   /* invalid argument (sizes, symmetry, start determinant) */
#define CDFCI_ERR_NONFINITE     -2   /* NaN/Inf in the integrals or in a step */
#define CDFCI_ERR_TABLE_FULL    -3   /* stored determinants exceed max_load * capacity, or probe limit hit */
#define CDFCI_ERR_TIMEOUT       -4   /* a bounded device wait gave up */
#define CDFCI_ERR_CUDA          -5   /* a CUDA runtime call failed */
#define CDFCI_ERR_UNIMPLEMENTED -6   /* entry point not available for this kind of handle */
#define CDFCI_ERR_NOMEM         -7   /* host or device allocation failed */
#define CDFCI_ERR_CAPACITY      -8   /* caller's output buffer too small (required size returned) */
#define CDFCI_ERR_NOT_NEGATIVE  -9   /* reduced problem has no negative eigenvalue (needs E0 < 0) */
#define CDFCI_ERR_INTERNAL     -10   /* a device-side consistency check failed (the access was skipped) */

typedef struct cdfci_ctx *cdfci_handle;

/*
 * Solver options (Sec. "Example Usage", JSON block solver/cdfci; Sec.
 * "Solvers for Ground and Excited States" for the stopping rule).
 */
typedef struct {
    int32_t  num_coordinates;  /* m: 1 = CDFCI (Alg. 1), 2..1023 = mCDFCI (Alg. 2) */
    int32_t  log2_capacity;    /* hash table holds 2^log2_capacity slots of 32 bytes */
    double   z_threshold;      /* tau of the compression rule (Sec. CDFCI); 0 = none */
    double   max_load;         /* stored determinants <= max_load * capacity (default 0.79) */
    double   dx_damping;       /* theta of the damped accumulator d <- theta d + (1-theta)|eta| */
    double   dx_threshold;     /* stop once d < this (0 = run the requested iterations) */
    uint64_t ref_alpha;        /* start determinant {A, B}; both 0 = aufbau on h_pp */
    uint64_t ref_beta;
    int32_t  block_threads;    /* reserved (the kernels' block sizes are fixed); ignored */
    int32_t  grid_blocks;      /* m = 1: CTAs that evaluate one column (0 = sized from the column
                                  length: about 256 elements per CTA, at most 64 CTAs).  Up to 16 they form one
                                  thread-block cluster (rounded to a size that can be resident);
                                  above 16 the loop runs as one cooperative grid of that many CTAs
                                  (at most the number that can be co-resident, clamped) whose CTAs
                                  hand their partials over once per iteration through round-numbered
                                  words in device memory (bounded waits); m > 1: ignored */
    int32_t  graph_chunk;      /* m = 1: iterations per persistent launch (0 = 65536);
                                  m > 1: iterations per captured CUDA graph (0 = 8) */
    int32_t  deterministic;    /* reserved.  m = 1 is deterministic (fixed-order reductions, one update
                                  per b_j per iteration); m > 1 adds several columns' contributions to
                                  one b_j with FP64 atomics, whose order (last-bit rounding) can vary */
    void    *cuda_stream;      /* cudaStream_t the work is queued on; NULL = a library stream */
    int32_t  num_states;       /* K + 1: 1 = ground state; 2..8 = xCDFCI (Alg. 3, Sec. "Coordinate-Descent
                                  Methods for Excited States") for the K + 1 lowest states, with
                                  num_coordinates = 1.  Start rows: the reference determinant and the K
                                  determinants of its column with the lowest diagonal H_DD (ties: the
                                  smaller key), C = [e_{D_0} .. e_{D_K}] */
    int32_t  z_threshold_search; /* 1: the r-th tenfold raise of tau comes when the stored determinants
                                  pass 1 - 2^-(r+1) of max_load * capacity (50 %, 75 %, 87.5 %, ...),
                                  the first from at least 1e-6 |E|; checked between launches, so a run
                                  that would fill the table continues with stronger compression (Sec.
                                  "Example Usage": adjust compression to fit the memory); tau never
                                  decreases; the current tau is in cdfci_stats.z_threshold */
    double   max_memory;       /* > 0: GiB for the wavefunction's table (and xCDFCI rows): log2_capacity
                                  becomes the largest that fits; 0 = use log2_capacity */
    int32_t  integral_symmetry; /* 8 (or 0, the default): real orbitals, g has the 8-fold symmetry and every
                                  image is canonicalised; 4: g is real with (pq|rs) = (rs|pq) = (qp|sr)
                                  only, as for the plane-wave orbitals of the k-space Hubbard model
                                  (HamiltonianHubbardK of Sec. "The Hamiltonian Class": (pq|rs) =
                                  (U/L) delta(k_q - k_p + k_s - k_r)); g is then validated against those
                                  two symmetries and used as given.  The kernels read doubles as
                                  (ia|jb) with i, j occupied in the column's determinant and a, b in the
                                  row's, and diagonals as J_pq = (pp|qq), K_pq = (pq|qp), so both forms
                                  give Eq. (entry).  cdfci_gradient's dE/dg assumes the 8-fold form */
} cdfci_params;

/* Progress report (the console row of Sec. "Expected Console Output"). */
typedef struct {
    int64_t iterations;        /* completed coordinate (block) updates */
    double  energy;            /* alpha / mu: Rayleigh-quotient estimate (Alg. 1/2, last line) */
    double  mu;                /* c^T c (leading double of the double-double value) */
    double  alpha;             /* c^T H c accumulated by Eq. (update-var) (leading double) */
    double  dx;                /* damped step accumulator */
    int64_t nnz_c;             /* |x|_0: stored coefficients that are nonzero */
    int64_t n_slots;           /* |z|_0: determinants stored in the table */
    int64_t last_column;       /* |H_i|_0: nonzero elements of the last processed column(s) */
    int64_t elements;          /* cumulative nonzero H elements evaluated by column updates */
    int64_t applied;           /* ... of which passed the compression rule and updated b */
    int64_t dropped;           /* ... of which were dropped by the compression rule */
    int64_t inserted;          /* cumulative new table entries */
    double  load;              /* n_slots / capacity */
    int32_t status;            /* sticky device status (0 or a CDFCI_ERR_* code) */
    int32_t converged;         /* 1 once dx < dx_threshold */
    int64_t reduced_iterations;/* m > 1: cumulative iterations of the reduced eigensolver (0 for m = 1) */
    int32_t grid_blocks;       /* m = 1: CTAs that evaluate a column (as resolved); 0 for m > 1 */
    int32_t grid_wide;         /* m = 1: 1 if they run as a cooperative grid (more than a cluster holds) */
    double  z_threshold;       /* the tau in force (changes only under z_threshold_search) */
} cdfci_stats;

/* Fills *p with the defaults (m = 1, 2^22 slots, tau = 0, max_load = 0.79,
   theta = 0.9, no early stop, aufbau start, deterministic). */
void cdfci_default_params(cdfci_params *p);

/*
 * Build a solver: copies h and g to the device, allocates the hash table,
 * and performs the initialisation of Algorithms 1 and 2: c = e_ref,
 * b = H c (one column, compression applied), mu = 1, alpha = H_ref,ref, the
 * candidate set = that column.  The start determinant is params->ref_{alpha,
 * beta} or, when both are 0, the aufbau determinant of h_pp (smallest
 * diagonal first, ties to the lower index) standing in for the Hartree-Fock
 * reference of Sec. "Example Usage".
 * Errors: CDFCI_ERR_ARG (N, n_alpha, n_beta out of range, a start key with
 * the wrong electron counts, asymmetric h or g), CDFCI_ERR_NONFINITE,
 * CDFCI_ERR_NOMEM, CDFCI_ERR_CUDA.  *out is NULL on failure.
 */
int cdfci_create(const double *h, const double *g, int N, int n_alpha, int n_beta,
                 const cdfci_params *params, cdfci_handle *out);

/*
 * The k-space Hubbard model (HamiltonianHubbardK of Sec. "The Hamiltonian
 * Class": a D-dimensional periodic orthogonal lattice, nearest-neighbour
 * hopping t, on-site U) in plane-wave orbitals, one per momentum (row-major
 * momentum indices n, the last direction fastest; k_d = 2 pi n_d / shape[d]).
 * h = diag(eps_k), eps_k = sum_d -2t cos k_d over directions of extent >= 3,
 * -t cos k_d for extent 2 (a single bond), rounded to 12 decimals; (pq|rs) =
 * U/L when k_q - k_p + k_s - k_r = 0, else 0 (integral_symmetry = 4 is
 * implied).  The handle also keeps the lattice's momentum tables, so the
 * column enumeration drops the opposite-spin doubles that do not conserve
 * momentum before any integral or table access.  shape: D extents (host),
 * prod(shape) <= 64 orbitals; otherwise as cdfci_create.
 */
int cdfci_create_hubbard_k(const int32_t *shape, int32_t D, double t, double U, int n_alpha, int n_beta,
                           const cdfci_params *params, cdfci_handle *out);

/*
 * Run n_iter iterations of Algorithm 1 (m = 1: Gauss-Southwell choice over the
 * last column, Eq. choose-i; exact line search, appendix; Eq. update-var with
 * compression; recalculation of b_i, Eq. recalculate-b) or Algorithm 2
 * (m > 1: top-m choice, Eq. choose-I; (m+1)-dimensional reduced eigenproblem;
 * c <- gamma c + E_I eta, b <- gamma b + H_{:,I} eta; recalculation of b_I).
 * Work is queued on the handle's stream; the call returns after the stats
 * are copied back (stats may be NULL).  Stops early once dx < dx_threshold.
 */
int cdfci_step(cdfci_handle h, int64_t n_iter, cdfci_stats *stats);

/*
 * Energy of the current vector: mode 0 = alpha / mu (double-double ratio,
 * Alg. 1 last line); mode 1 = exact Rayleigh quotient sum_i c_i (Hc)_i / c.c
 * recomputed from the stored c with fresh columns (independent of b).
 */
int cdfci_energy(cdfci_handle h, int mode, double *E);

/*
 * The exact Rayleigh quotient c^T H' c / c^T c of the handle's stored vector c
 * under other integrals h1 (N*N) and g2 (N^4, (pq|rs)) of the same orbital
 * space and electron counts (host or device pointers, copied; validated as by
 * cdfci_create with the handle's integral_symmetry): the energy of a fixed
 * state in another Hamiltonian, as the orbital subproblem of Sec. "Optimal
 * Orbital Selections" evaluates the fixed FCI state in rotated orbitals.  Used
 * for central differences of the energy along any integral direction; the
 * handle's state is not changed.  E: host.  Errors: CDFCI_ERR_ARG,
 * CDFCI_ERR_NONFINITE, CDFCI_ERR_NOMEM, CDFCI_ERR_UNIMPLEMENTED (xCDFCI).
 */
int cdfci_energy_with(cdfci_handle h, const double *h1, const double *g2, double *E);

/*
 * get_column of Sec. "The Hamiltonian Class": all (D', H_{D',D}) with a
 * nonzero FP64 value (Eq. entry), diagonal included, as an unordered list.
 * key = {A, B} (host or device, 2 words).  keys_out (2 words per entry) and
 * vals_out hold up to cap entries; *n_out receives the column length (host
 * pointer).  Returns CDFCI_ERR_CAPACITY when cap is too small (nothing written).
 */
int cdfci_get_column(cdfci_handle h, const uint64_t *key, uint64_t *keys_out, double *vals_out,
                     int64_t cap, int64_t *n_out);

/*
 * get_entry and get_diagonal of Sec. "The Hamiltonian Class": one element
 * H_{row, col} of Eq. (entry) (0.0 beyond a double excitation) and the
 * diagonal H_{key, key}.  Keys are {A, B} (host or device, 2 words each) with
 * the handle's N and electron counts (else CDFCI_ERR_ARG); *value is a host
 * pointer.  H is symmetric, so the order of the two keys does not matter.
 */
int cdfci_get_entry(cdfci_handle h, const uint64_t *row_key, const uint64_t *col_key, double *value);
int cdfci_get_diagonal(cdfci_handle h, const uint64_t *key, double *value);

/*
 * All stored determinants with their true (unscaled) c and b values, in
 * table order.  keys (2 words per entry), c, b hold up to cap entries (c or b
 * may be NULL); *n_out = number stored.  CDFCI_ERR_CAPACITY if cap is too small.
 */
int cdfci_export(cdfci_handle h, uint64_t *keys, double *c, double *b, int64_t cap, int64_t *n_out);

/*
 * xCDFCI handles (num_states = K + 1 > 1): the K + 1 energies, ascending, from
 * the pencil (C^T H C, C^T C) of the current rows (the generalised eigenvalue
 * problem that closes Alg. 3); *n_out = K + 1 (1 and the Rayleigh quotient for
 * other handles).  CDFCI_ERR_CAPACITY if cap < K + 1.
 */
int cdfci_energies(cdfci_handle h, double *E, int32_t cap, int32_t *n_out);

/*
 * Per-kernel device time of the mCDFCI iteration (Alg. 2; handles with
 * num_coordinates > 1): runs n_iter iterations of the solve (they advance it
 * like cdfci_step) launch by launch instead of as a graph, with a CUDA event
 * recorded before every launch on the handle's stream, and writes into ms the
 * milliseconds spent from each launch to the next, summed over the
 * iterations, in launch order: 0 choice keys + level-0 histogram, 1 level-1
 * histogram and the levels below it, 2 collect, 3 exact ties and the sort of
 * the chosen set, 4 c_I / b_I / H_II, 5 reduced problem, 6 scatter of the m
 * columns, 7 b_I recalculated.  *n_kernels = 8 (host pointer); ms holds up to
 * cap values (host pointer).  CDFCI_ERR_CAPACITY if cap < 8,
 * CDFCI_ERR_UNIMPLEMENTED for other handles.
 */
int cdfci_time_kernels(cdfci_handle h, int64_t n_iter, double *ms, int32_t cap, int32_t *n_kernels);

/*
 * Measurement only; the paper has no counterpart.  The memory system's rate
 * for the hash scatter's access pattern (Sec. "Parallelization Support": the
 * update is bound by irregular hash-table accesses): n_ops operations, each
 * on a pseudo-random slot (SplitMix64 of seed + op) of a table of
 * 2^log2_slots 32-byte slots {A, B, c, b}: one 32-byte load of the slot and
 * an FP64 add to b whose result is not read (the scatter's lookup of an
 * existing key).
 * Operations are independent, so every lane keeps several in flight: the rate
 * bounds any lookup sequence of random slots from above.  table (device, 32-byte
 * aligned, 2^log2_slots * 32 bytes, caller-owned) must be larger than L2 for
 * the rate to be DRAM's; its b fields are changed, nothing else is written.
 * The launch is queued on cuda_stream (a cudaStream_t, NULL = legacy default)
 * and the call returns at once; time it with events on that stream.
 * Errors: CDFCI_ERR_ARG (NULL or misaligned table, log2_slots outside
 * [10, 34], n_ops < 0), CDFCI_ERR_CUDA.
 */
int cdfci_probe_slots(void *table, int log2_slots, int64_t n_ops, uint64_t seed, void *cuda_stream);

/*
 * Degenerate-subspace start (the k-space Hubbard example of the paper's
 * numerical section: when the lowest one-body configurations are degenerate,
 * H restricted to all of them is diagonalised and its lowest eigenvector is
 * the start).  The one-body energies are the diagonal h_pp; per spin the
 * lowest shells are filled, and the last, partly filled shell (levels within
 * tol * max(1, |level|), tol <= 0: 1e-10) contributes every choice of its
 * remaining electrons.  The set S (alpha choices x beta choices, ordered by the
 * 128-bit key (B << 64) | A) must hold at most cap determinants (cap <= 0:
 * 1024); H_SS comes from this handle's columns, its eigenpairs from cyclic
 * Jacobi rotations on the host (a one-time start, |S| x |S| dense).  When the
 * lowest eigenvalue is degenerate (eigenvalues within 1e-9 of it, relative;
 * 4-fold at the paper's 4x4 half filling, over two total-momentum sectors)
 * every vector of its eigenspace is an eigenvector: the start is the
 * projection onto that eigenspace of the ramp r_s = 1 + s / |S| (s = position
 * in S), which has a component in every momentum sector of it (one basis
 * vector may lie in a single sector, and H conserves momentum, so the
 * iteration could never reach the ground state's sector).  For a simple
 * eigenvalue this is its eigenvector.  The vector is normalised with its
 * largest component positive (ties: the first in S).  The vector then replaces the
 * state as cdfci_set_initial would (zero components skipped).  *n_det = |S|,
 * *E_sub = the lowest eigenvalue (host pointers; E_sub may be NULL).
 * CDFCI_ERR_CAPACITY if |S| > cap (*n_det set), CDFCI_ERR_UNIMPLEMENTED for
 * xCDFCI handles.
 */
int cdfci_set_initial_degenerate(cdfci_handle h, double tol, int64_t cap, int64_t *n_det, double *E_sub);

/*
 * The degenerate set alone (host only, no handle, no device work): the
 * determinants of lowest one-body energy for the levels eps[0..N) (host),
 * built and ordered as cdfci_set_initial_degenerate builds S.  keys (host, 2
 * words per determinant, {A, B}) receives them when not NULL (room for cap);
 * *n_det = |S|.  CDFCI_ERR_CAPACITY if |S| > cap (with keys NULL, cap <= 0
 * means 1024), CDFCI_ERR_ARG for N, electron counts or levels out of range,
 * or for keys given with cap <= 0.
 */
int cdfci_degenerate_set(const double *eps, int N, int n_alpha, int n_beta, double tol, int64_t cap,
                         uint64_t *keys, int64_t *n_det);

/*
 * All stored determinants with their rows C_{D,:} and B_{D,:} = (HC)_{D,:}
 * (num_states values each, row-major), in table order; for other handles the
 * same as cdfci_export (one value each).  CDFCI_ERR_CAPACITY if cap is too small
 * (*n_out = number stored).  The columns of C span the K + 1 lowest eigenvectors
 * at convergence; they are not orthonormal (Sec. "Coordinate-Descent Methods
 * for Excited States": the pencil gives the eigenvectors).
 */
int cdfci_export_states(cdfci_handle h, uint64_t *keys, double *C, double *B, int64_t cap, int64_t *n_out);

/*
 * OptOrbFCI (Alg. 4, Sec. "Optimal Orbital Selections"): N orbitals phi = psi U
 * chosen from M >= N by alternating the FCI problem in the current basis
 * (this library's solver with p->fci, p->inner_iterations steps) with the
 * orbital subproblem (eq. subopt): P4(U) = sum h'gamma + 1/2 sum g'Gamma over
 * the M x N matrices with orthonormal columns, the RDMs of the current FCI
 * state fixed, by p->bb_steps projected-gradient steps (eq. projBB)
 * U <- orth(U - t_k grad P4(U)) with alternating Barzilai-Borwein steps t_k =
 * <S,S>/|<S,Y>| (odd k) and |<S,Y>|/<Y,Y> (even k), t_0 = 0.1 / max(1, ||grad||_F),
 * orth = the polar factor (Newton-Schulz on the device); the U with the lowest
 * P4 met is kept.  h (M x M), g (M^4, (pq|rs)) and U (M x N, row-major, in: a
 * start with orthonormal columns, out: the last basis) are host or device
 * pointers; energies (host) receives E_0 of each outer iteration's FCI solve
 * (p->outer values).  Every step runs on the device (integral transformation,
 * gradient, projection, reductions); the host only sequences them.  Errors:
 * CDFCI_ERR_ARG (sizes, U not orthonormal to 1e-10, num_states > 1), and those
 * of cdfci_create / cdfci_step.
 */
typedef struct {
    int32_t      outer;             /* outer iterations of Alg. 4 */
    int32_t      bb_steps;          /* projected-gradient steps of the orbital subproblem per outer iteration */
    int64_t      inner_iterations;  /* solver iterations per FCI problem */
    cdfci_params fci;               /* the inner solver (num_states = 1) */
} cdfci_optorb_params;
int cdfci_optorb(const double *h, const double *g, int M, int N, int n_alpha, int n_beta, double *U,
                 const cdfci_optorb_params *p, double *energies);

/*
 * Start vector (optional, replaces the state): c = sum_k c[k] e_{keys k},
 * keys 2 words per entry (A, B), n >= 1 distinct determinants with the
 * handle's N, n_alpha, n_beta and at least one nonzero c; host or device
 * pointers, copied.  The table is cleared and the entries are applied in the
 * given order as steps of Algorithm 1 (m = 1) or one-coordinate block steps
 * (m > 1) from c = 0 with the step fixed to c[k]: each column is scattered
 * with the compression rule of Sec. 3.1, so b = Hc as that rule accumulates it,
 * mu = c.c and alpha = c.Hc (double-double, Eq. update-var); the reference
 * start of cdfci_create is the case n = 1, c = 1.  The next cdfci_step then
 * chooses among the entries of the last start column and that coordinate
 * (m = 1) or among every entry the start columns touched (m > 1).  These steps
 * are not counted as iterations.  A sticky error status is cleared.  For m > 1
 * at most m entries (their columns' candidates must fit the candidate list).
 * Errors: CDFCI_ERR_ARG (a key outside N or with the wrong electron counts, a
 * repeated key, all c zero, a NaN, n out of range), CDFCI_ERR_TABLE_FULL,
 * CDFCI_ERR_NOMEM, CDFCI_ERR_CUDA.
 */
int cdfci_set_initial(cdfci_handle h, const uint64_t *keys, const double *c, int64_t n);

/*
 * Checkpoint / resume (the paper's solver can stop and later continue from
 * a saved wavefunction, Sec. "Solvers for Ground and Excited States"; it
 * gives no format).  A checkpoint is this
 * header plus n_entries rows (keys: 2 words; c, b: as stored, i.e. divided by
 * the scale s for m > 1; flags: bit 0 = a candidate of the next block
 * selection).  cdfci_checkpoint fills *hdr and then, if cap >= n_entries, the
 * rows (host or device pointers; flags may be NULL); a smaller cap returns
 * CDFCI_ERR_CAPACITY with *hdr filled, so a caller can size its arrays.  The
 * m = 1 state between steps includes the partial results of the last column
 * (its best candidate, the gather sum behind the recalculated b of Eq.
 * recalculate-b, counters); they are stored folded into one, in the order the
 * next step would fold them, so on a handle with any grid_blocks the next
 * step is the one the writer would take, and with the same grid_blocks every
 * following step is bit for bit the same (another grid folds later columns'
 * gather sums in another order: agreement to the last bits).  m > 1 adds
 * several columns' contributions to one b_j with FP64 atomics, so its
 * continuation agrees to the last bits.  cdfci_restore needs a handle with the same N, n_alpha,
 * n_beta and the same kind of step (m = 1, or m > 1 with the candidates
 * fitting its candidate list); it clears the table, re-inserts the rows and
 * sets every scalar.  Errors: CDFCI_ERR_ARG (mismatch, bad header or keys,
 * duplicates), CDFCI_ERR_TABLE_FULL (the rows exceed this handle's max_load),
 * CDFCI_ERR_NOMEM, CDFCI_ERR_CUDA.
 */
typedef struct {
    int32_t  version;          /* 1 */
    int32_t  N, n_alpha, n_beta;
    int32_t  num_coordinates;  /* m of the handle that wrote it */
    int32_t  have_prev;        /* m = 1: a coordinate was processed and its column's partials are pending */
    int32_t  done;             /* the dx stopping rule has fired */
    int32_t  has_best;         /* m = 1: the pending column has a candidate */
    int64_t  n_entries;        /* rows that follow */
    double   mu[2], alpha[2];  /* double-double c.c and c.Hc (hi, lo) */
    double   scale[2];         /* m > 1: double-double scale s of the stored values (1 for m = 1) */
    double   dx, energy, last_gamma;
    int64_t  iterations, nnz_c, n_slots, elements, applied, dropped, inserted, last_column, reduced_iterations;
    /* m = 1: the coordinate processed last */
    uint64_t prev_key[2];
    double   prev_c, prev_Hii, prev_eta, prev_mu_g;
    /* m = 1: the pending column folded (best candidate by |b + mu c| bits, gather sum, counters) */
    uint64_t best_key[2];
    uint64_t best_gbits;
    double   best_b, best_c, gather;
    int64_t  pending[4];       /* elements, applied, dropped, inserted of the pending column */
    int32_t  pending_err;
    int32_t  reserved;
} cdfci_checkpoint_header;
int cdfci_checkpoint(cdfci_handle h, cdfci_checkpoint_header *hdr, uint64_t *keys, double *c, double *b, uint8_t *flags,
                     int64_t cap);
int cdfci_restore(cdfci_handle h, const cdfci_checkpoint_header *hdr, const uint64_t *keys, const double *c, const double *b,
                  const uint8_t *flags);

/*
 * The coordinates chosen by the most recent iteration and their step sizes
 * (eta, in true units), up to cap entries; *m_out receives the count.
 */
int cdfci_last_step(cdfci_handle h, uint64_t *keys, double *eta, int64_t cap, int64_t *m_out);

/*
 * Spin-summed reduced density matrices of the current vector, normalised by
 * c.c (Sec. "Optimal Orbital Selections"):
 *   rdm1[p*N+q]               = gamma_pq   = sum_s  <a+_ps a_qs>
 *   rdm2[((p*N+q)*N+r)*N+s]   = Gamma_pqrs = sum_st <a+_ps a+_rt a_st a_qs>
 * in chemists' order, so that E = sum h_pq gamma_pq + 1/2 sum (pq|rs) Gamma_pqrs.
 * rdm1 (N*N doubles) and rdm2 (N^4 doubles, or NULL) are host or device memory.
 * Cost: one pass over the stored determinants, each enumerating all its
 * single and double excitations with a table lookup per excitation.
 */
int cdfci_rdm(cdfci_handle h, double *rdm1, double *rdm2);

/*
 * Derivatives of the energy E = sum h gamma + 1/2 sum (pq|rs) Gamma of the
 * current vector (Hellmann-Feynman at convergence): dE_dh = gamma (N*N),
 * dE_dg = 1/2 Gamma averaged over the 8-fold symmetry of (pq|rs) (N^4: the
 * derivative along 8-fold symmetric perturbations), dE_dkappa = 2 (F - F^T)
 * (N*N, antisymmetric) for orbitals rotated by U = exp(kappa),
 * F_pq = sum_r h_pr gamma_qr + sum_rst (pr|st) Gamma_qrst, so that
 * dE = 1/2 sum_pq dE_dkappa[p][q] dkappa_pq.  h and g are the handle's
 * (symmetrised) integrals.  Any output may be NULL; host or device memory.
 */
int cdfci_gradient(cdfci_handle h, double *dE_dh, double *dE_dg, double *dE_dkappa);

/*
 * Batches: many independent solvers (problems of different sizes: molecules,
 * lattices) stepped together; cdfci_batch_step(n_iter) runs n_iter iterations
 * of every problem (Algorithm 1 for num_coordinates = 1, Algorithm 2 with its
 * own m otherwise).
 *   m = 1 solvers: one persistent launch (replayed from a captured CUDA
 *   graph) runs them all, one thread-block cluster per problem, with no
 *   communication between clusters; they need the same grid_blocks (CTAs per
 *   problem, at most 16: a grid-wide handle is rejected).
 *   m > 1 solvers: one captured CUDA graph holds graph_chunk iterations of
 *   every such problem, each problem's iteration kernels (with its own launch
 *   shapes and block size m) on a branch of its own, forked from the batch's
 *   stream and joined back, so that the problems run side by side; one graph
 *   launch advances them all.  z_threshold_search is applied per problem
 *   between graph launches (the graph is captured again when a tau moves).
 * Each problem's arithmetic is exactly its solo step's.  The batch does not
 * own the handles, which must outlive it and not be num_states > 1; while
 * batched they are queued on the first handle's stream.  A handle stays usable
 * on its own: cdfci_step continues from the batch's state.  stats (n entries,
 * in the order of hs, or NULL) receives every problem's report; the return
 * code is the first error, if any.
 */
typedef struct cdfci_batch *cdfci_batch_handle;
int cdfci_batch_create(const cdfci_handle *hs, int n, cdfci_batch_handle *out);
int cdfci_batch_step(cdfci_batch_handle b, int64_t n_iter, cdfci_stats *stats);
void cdfci_batch_destroy(cdfci_batch_handle b);

/*
 * Autotuner: picks the block size m (num_coordinates) and, for m = 1, the CTAs
 * per column (grid_blocks, the CTAs that evaluate one determinant's
 * column) that reach a given energy soonest on this problem (a
 * proxy for time-to-E).  All candidates start from the same point.  First m =
 * 1 with the configured grid_blocks (0 = sized from the column) runs for an
 * equal share of `seconds`, and the energy it reaches is the target.  Then m
 * = 1 with grid_blocks in {1, 2, 4, 8, 16, 32, 64, 128} (the trajectory is the same, only
 * the speed differs) and m in {4, 16, 64, 256} (at most the library's limit)
 * each run until they reach the target or twice the share has passed.  The
 * time spent in cdfci_step is what counts.  On return params->num_coordinates
 * and params->grid_blocks hold the fastest; report (may be NULL) receives
 * every candidate's m, grid_blocks, iterations, seconds, energy drop and score
 * (seconds to the target, -1 if not reached) and the index of the winner.
 * Errors as for cdfci_create; a candidate whose table fills up is scored by
 * what it reached before.
 */
typedef struct {
    int32_t n;                 /* candidates tried */
    int32_t chosen;            /* index of the winner */
    int32_t m[16];
    int32_t grid_blocks[16];   /* CTAs per column for m = 1 (as resolved by the library); 0 for m > 1 */
    int64_t iterations[16];
    double  seconds[16];
    double  energy_drop[16];   /* Hartree */
    double  score[16];         /* seconds to the target energy, -1 if not reached */
} cdfci_tune_report;
int cdfci_autotune(const double *h, const double *g, int N, int n_alpha, int n_beta, cdfci_params *params,
                   double seconds, cdfci_tune_report *report);

/* Current stats without running an iteration. */
int cdfci_get_stats(cdfci_handle h, cdfci_stats *stats);

/*
 * get_column without any device allocation, for callers that cannot call
 * cudaMalloc (code running inside a memory pool or allocator it does not own,
 * or a framework that forbids allocation on its hot path).  The paper has no
 * counterpart: it is the cdfci_get_column operation without a handle.
 *
 * h (N*N) and g (N^4) must be device memory, as must keys_out (2 words per
 * entry) and vals_out when cap > 0; key ({A, B}) may be host or device memory;
 * *n_out (host) receives the column length.  h and g are used exactly as
 * given: h must be symmetric and g exactly 8-fold symmetric for bit-for-bit
 * agreement with cdfci_get_column (whose handle symmetrises h and
 * canonicalises g at creation), and neither is checked for symmetry or for
 * NaN/Inf entries.
 * Work is queued on cuda_stream (a cudaStream_t; NULL = legacy default
 * stream) and the call waits for it: it reads the key and the column length
 * back to the host.  On a stream that is being captured it therefore returns
 * CDFCI_ERR_ARG before touching the stream, so the caller's capture stays
 * valid.
 * Scratch: a fixed array of about 80 KB inside the library image (counter,
 * J/K tables, pair tables), held by every GPU that loads the library until
 * the process exits.  Limit: N <= 63 orbitals; larger N is rejected with
 * CDFCI_ERR_ARG.  The first call on a device looks up the array's device
 * address and keeps it for that device; make that first call before any
 * stream capture.  The kept address belongs to the device context of that
 * first call: after cudaDeviceReset on that device it is stale, so the
 * function must not be called again in that process.  All calls on a device
 * share the array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Every call clears the
 * counter and rewrites the tables it reads, so nothing of an earlier call's
 * contents reaches its result.
 * Errors: CDFCI_ERR_ARG (sizes, host memory where device memory is needed,
 * a key with the wrong electron counts, a capturing stream),
 * CDFCI_ERR_CAPACITY (*n_out holds the required size; the buffers then hold
 * an unspecified part of the column), CDFCI_ERR_CUDA.
 */
int cdfci_column_noalloc(const double *h, const double *g, int N, int n_alpha, int n_beta, const uint64_t *key,
                         uint64_t *keys_out, double *vals_out, int64_t cap, int64_t *n_out, void *cuda_stream);

/*
 * FCIDUMP ingestion (Sec. "Example Usage": the molecular Hamiltonian is read
 * from an FCIDUMP file, "fcidump_path", with a "threshold" below which
 * integral values are neglected).  Host code only; no device work.
 *
 * cdfci_fcidump_header reads the namelist header "&FCI NORB=.., NELEC=..,
 * MS2=.., ... &END" (or "/" as the end): *norb = N, *nelec, *ms2 = 2 S_z
 * (0 when absent), so n_alpha = (nelec + ms2) / 2, n_beta = (nelec - ms2) / 2.
 *
 * cdfci_fcidump_read fills h (N*N, row-major, host) and g (N^4, (pq|rs)
 * row-major, host) from the integral lines "value i j k l" (1-based): i j k l
 * all > 0 set (ij|kl) and its 8 symmetric images; k = l = 0 sets h_ij and h_ji;
 * i = j = k = l = 0 gives the core energy (*e_core, host, may be NULL; a
 * constant that the solver's energies do not include); i > 0, j = k = l = 0
 * lines (orbital energies) are skipped.  Entries absent from the file are 0.
 * A value with |value| < threshold is stored as 0 (threshold = 0 keeps all;
 * the core energy is never truncated).  Fortran exponents (1.0D-03) are
 * accepted.  norb must equal the header's NORB.  The caller owns h and g.
 * Errors: CDFCI_ERR_ARG (unreadable file, malformed header or line, an index
 * outside [0, N], N outside [1, 63], inconsistent NELEC/MS2, norb mismatch),
 * CDFCI_ERR_NONFINITE (a NaN or infinite value).
 */
int cdfci_fcidump_header(const char *path, int *norb, int *nelec, int *ms2);
int cdfci_fcidump_read(const char *path, double threshold, int norb, double *h, double *g, double *e_core);

/* Frees everything the handle owns (safe on NULL). */
void cdfci_destroy(cdfci_handle h);

/* Message of the last failure on this thread ("" if none). */
const char *cdfci_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CDFCI_H */
