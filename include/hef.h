/*
 * hef.h -- C ABI of the GB300 hyperedge effective-resistance library.
 *
 * The library computes the hyperedge effective-resistance estimates of
 * HyperEF 2.0 (arXiv 2511.06600, Algorithm 1, Section III-A.3) on one
 * NVIDIA GB300 (sm_103a):
 *
 *   1. hef_build_incidence   Algorithm 1 steps 1-2: the star expansion G_b
 *                            and clique expansion G_c of H = (V, E, w), kept
 *                            implicit as edge-major and vertex-major incidence.
 *   2. hef_krylov_basis      Algorithm 1 step 3, Eq. krylov: Krylov vectors
 *                            A x ... A^k x of both expansions' random-walk
 *                            operators from S random starts each.
 *   3. hef_orthonormalize    Algorithm 1 step 4: orthonormal basis of the
 *                            vertex parts (CholQR2, FP64 Cholesky).
 *   4. hef_edge_resistance   Algorithm 1 steps 5 and 7, Eqs. non-linerQ,
 *                            ratios and R: R_e = max_i spread_e(chi_i)^2 /
 *                            Q_H(chi_i).
 *
 * Conventions shared by every call
 *  - All array arguments are DEVICE pointers unless stated otherwise; the
 *    caller owns them and keeps them alive until the work on `stream` is done.
 *    `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *    asynchronous on `stream` and performs no host<->device synchronisation,
 *    except hef_incidence_check, which synchronises `stream`.
 *  - The library never allocates device memory.  Each call that needs
 *    scratch takes a caller-provided `workspace` of at least the size that
 *    its *_workspace_bytes query returns (256-byte aligned base).
 *  - Matrices are row-major: row r of an n x K matrix starts at r * ld
 *    elements; ld >= K.  Rows must start 16-byte aligned (ld * element size
 *    a multiple of 16 bytes).
 *  - Element types: HEF_F64 (double), HEF_F32 (float), HEF_BF16 (the basis
 *    V / Q stored as bfloat16, arithmetic in FP32 / FP64 as stated per call).
 *  - Return value: HEF_OK or a negative hef_status; hef_last_error() gives a
 *    thread-local message for the last failing call.  Errors found by device
 *    code (malformed incidence, non-positive weights) are recorded in the
 *    incidence's device status word: later kernels that use that incidence
 *    do no work, and hef_incidence_check returns HEF_ERR_INVALID_INPUT.
 */
#ifndef HEF_H_
#define HEF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hef_status;

#define HEF_OK 0
#define HEF_ERR_INVALID_ARG (-1)   /* host-side argument check failed */
#define HEF_ERR_CUDA (-2)          /* a CUDA launch or runtime call failed */
#define HEF_ERR_WORKSPACE (-3)     /* workspace missing, misaligned or too small */
#define HEF_ERR_BREAKDOWN (-4)     /* orthonormalisation lost every column */
#define HEF_ERR_TIMEOUT (-5)       /* a bounded device wait expired */
#define HEF_ERR_UNSUPPORTED (-6)   /* valid request outside supported sizes */
#define HEF_ERR_INVALID_INPUT (-7) /* device-side check of the hypergraph failed */
#define HEF_ERR_BOUNDS (-8)        /* HEF_DEBUG build: an index read from the
                                      incidence lay outside its array */

#define HEF_F64 0
#define HEF_F32 1
#define HEF_BF16 2 /* basis stored in BF16 (Krylov chains, Gram and spreads in
                      FP32; Cholesky and Q_H in FP64); K <= 511; no backward */

/* Reductions over basis vectors in hef_edge_resistance. */
#define HEF_REDUCE_MAX 0 /* Eq. R: R_e = max_i r_e(chi_i) */
#define HEF_REDUCE_SUM 1 /* sum_i r_e(chi_i); with Laplacian eigenvectors of a
                            2-pin graph as the basis this is Eq. eff_resist0 */
#define HEF_REDUCE_EMBED 2 /* Eq. R with p, q of Eq. ratios the pins farthest
                              apart in the whole K-dimensional embedding (one
                              pair per hyperedge; see hef_edge_resistance) */

/* Krylov pools (hef_krylov_basis_ops). */
#define HEF_OPS_CLIQUE 1 /* clique expansion only */
#define HEF_OPS_STAR 2   /* star expansion only: the earlier HyperEF pool */
#define HEF_OPS_BOTH 3   /* both (the mixed pool of Section III-A.3) */

/* Clique-expansion pair weight (Section III-A.3). */
#define HEF_CLIQUE_HYPEREDGE 0 /* w(e)/(|e|-1): clique degree = hypergraph degree */
#define HEF_CLIQUE_PAPER 1     /* w(e)/C(|e|,2): weight spread evenly over pairs */

/* Bits of the device status word (hef_incidence_check's detail output). */
#define HEF_BAD_EPTR 1u      /* eptr[0] != 0, eptr[m] != P or decreasing */
#define HEF_BAD_PIN 2u       /* a pin outside [0, n) */
#define HEF_DUP_PIN 4u       /* a vertex repeated within one hyperedge */
#define HEF_BAD_WEIGHT 8u    /* a weight that is not finite and > 0 */
#define HEF_WAIT_TIMEOUT 16u /* a bounded grid-wide wait of the one-launch
                                Krylov form expired (hef_incidence_check then
                                returns HEF_ERR_TIMEOUT) */
#define HEF_BOUNDS 32u       /* HEF_DEBUG build: a kernel read a vertex or
                                hyperedge index outside [0, n) or [0, m) from
                                the incidence; the access was redirected to
                                index 0 and hef_incidence_check returns
                                HEF_ERR_BOUNDS */

const char* hef_last_error(void);

const char* hef_status_string(hef_status s);
int32_t hef_abi_version(void);

/* ------------------------------------------------------------------------
 * Launch accounting and kernel timing (no counterpart in the paper: this is
 * the library's tracing facility).
 *
 * hef_launch_count: number of kernels this library has launched in the
 * process so far (all threads).
 * hef_trace_kernels: from now on, record a pair of CUDA events on the launch
 * stream around every launch of a library kernel whose name contains
 * `name_substring` (e.g. "k_score_pass"); NULL or "" stops recording.  At most
 * 65536 launches are recorded between reads.
 * hef_trace_read: synchronises the recorded events, writes per kernel name
 * (up to `cap` names, 64 chars each, NUL-terminated) the number of launches
 * and their summed duration in ms, forgets the records, and returns the number
 * of distinct names recorded.
 * ---------------------------------------------------------------------- */
uint64_t hef_launch_count(void);
hef_status hef_trace_kernels(const char* name_substring);
int32_t hef_trace_read(int32_t cap, char* names, int64_t* launches,
                       double* total_ms);

/* ------------------------------------------------------------------------
 * Incidence (Algorithm 1 steps 1-2; expansions of Section III-A.3).
 *
 * Input H = (V, E, w) in edge-major (CSC) form: hyperedge e has the pins
 * pins[eptr[e] .. eptr[e+1]) (vertex ids in [0, n), distinct within e) and
 * weight w[e] > 0.  0 <= n, m; 0 <= P = eptr[m] < 2^31.
 *
 * The build copies what it needs into `workspace` (CSC in a locality order of
 * the hyperedges, the vertex-major transpose, per-edge weights w/(|e|-1) or
 * w/C(|e|,2) and w/|e|, vertex degrees of both expansions), validates the
 * input on the device and records problems in the device status word.
 * Hyperedges with fewer than 2 pins join neither expansion and score 0.
 * The returned handle is a small host object (malloc); it refers to the
 * workspace, which must outlive it.  Free it with hef_free_incidence.
 * ---------------------------------------------------------------------- */
typedef struct hef_incidence hef_incidence;

size_t hef_incidence_workspace_bytes(int64_t n, int64_t m, int64_t P);

hef_status hef_build_incidence(int64_t n, int64_t m, int64_t P,
                               const int64_t* eptr, const int32_t* pins,
                               const double* w, int32_t clique_mode,
                               void* workspace, size_t workspace_bytes,
                               void* stream, hef_incidence** out);

/* Synchronises `stream` and returns HEF_ERR_INVALID_INPUT (with the status
 * bits in *detail, the first offending hyperedge in *where; either may be
 * NULL) if the device-side validation failed, HEF_ERR_TIMEOUT if a bounded
 * device wait of a later call on this incidence expired (HEF_WAIT_TIMEOUT),
 * HEF_ERR_BOUNDS if a kernel of the bounds-checked build met an index
 * outside its array (HEF_BOUNDS), else HEF_OK. */
hef_status hef_incidence_check(const hef_incidence* inc, void* stream,
                               uint32_t* detail, int64_t* where);

/* ------------------------------------------------------------------------
 * Bounds-checked build (no counterpart in the paper; a debugging aid).
 *
 * The library built with -DHEF_DEBUG=1 (libhef_debug.so: `python -m
 * paper_2511_06600_gb300.build --debug`) checks every vertex or hyperedge
 * index that a gather of the Krylov, scoring and backward kernels reads from
 * the incidence (pins, incidence lists) against its array before using it.
 * An index outside the array sets HEF_BOUNDS in the incidence's status word
 * and the access goes to index 0 instead, so the kernel never reads outside
 * its buffers; hef_incidence_check then returns HEF_ERR_BOUNDS.  The regular
 * build has no checks (the incidence build validates every pin).
 *
 * hef_debug_checks: 1 for the bounds-checked build, 0 otherwise.
 * hef_debug_set_pin: bounds-checked build only: overwrites pin slot `slot`
 *   (internal CSC order, 0 <= slot < P) of a built incidence with `value`
 *   (a copy on `stream`, which it synchronises), so that a test can plant an
 *   index that the checks must catch.  The regular build returns HEF_ERR_UNSUPPORTED and
 *   touches nothing; bad arguments give HEF_ERR_INVALID_ARG.
 * ---------------------------------------------------------------------- */
int32_t hef_debug_checks(void);
hef_status hef_debug_set_pin(const hef_incidence* inc, int64_t slot, int32_t value,
                             void* stream);

hef_status hef_incidence_sizes(const hef_incidence* inc, int64_t* n,
                               int64_t* m, int64_t* P);

/* Copies of the built incidence, for callers that consume the expansions
 * (e.g. a downstream clustering): perm[m] internal -> caller hyperedge id
 * (the locality order: ascending smallest pin, ties by caller id);
 * vptr[n+1] and vedge[P] the vertex-major incidence (caller hyperedge ids,
 * in locality order within each vertex); dc[n], db[n] the vertex degrees of
 * the clique and star expansions.  Any output may be NULL.  Asynchronous. */
hef_status hef_incidence_export(const hef_incidence* inc, int32_t* perm,
                                int32_t* vptr, int32_t* vedge, double* dc,
                                double* db, void* stream);

void hef_free_incidence(hef_incidence* inc);

/* ------------------------------------------------------------------------
 * Krylov basis (Algorithm 1 step 3, Eq. krylov; Section III-A.3).
 *
 * For each expansion op (0 = clique on n vertices, 1 = star on n + m
 * vertices) and start s < S, the chain x, M x, ..., M^k x of the random-walk
 * operator M = D^-1 W, started from the given random vector with the
 * trivial eigenvectors of M (the constant on non-isolated vertices, and for
 * the bipartite star expansion the vertex-side and star-side constants)
 * projected out in the degree-weighted inner product.  The raw start is not
 * part of the basis.  Vertex rows of the j-th chain vector (j = 1..k) go to
 * column c = (j-1)*2S + op*S + s of V (n x ldv, dtype), scaled arbitrarily
 * per column and not mean-free: hef_orthonormalize removes the mean and the
 * scale.  A chain whose Krylov space is exhausted yields zero columns.
 *
 * x0_clique: n x S row-major double.  x0_star: (n + m) x S row-major double,
 * vertex rows first, then one row per hyperedge in the caller's order.
 * K = 2 k S <= 512; S in {1, 2, 4, 8, 16}; ldv >= K.
 * ---------------------------------------------------------------------- */
size_t hef_krylov_workspace_bytes(const hef_incidence* inc, int32_t k,
                                  int32_t S, int32_t dtype);

hef_status hef_krylov_basis(const hef_incidence* inc, int32_t k, int32_t S,
                            int32_t dtype, const double* x0_clique,
                            const double* x0_star, void* V, int64_t ldv,
                            void* workspace, size_t workspace_bytes,
                            void* stream);

/* Launch form of the Krylov calls made from the calling host thread
 * (a library setting; the paper has no counterpart).  on = 1 (default): for
 * hypergraphs with n + m >= 32768 all k steps run as one cooperative launch
 * of one CTA per SM (smaller ones use the per-step form, which is as fast
 * there).  Each CTA owns a
 * balanced range of vertices and hyperedges, keeps their index lists in
 * shared memory across the steps, and meets the others at bounded grid-wide
 * barriers that carry the Lanczos reductions (a barrier that waits too long
 * sets HEF_WAIT_TIMEOUT in the incidence's status word instead of hanging).
 * The runtime starts a cooperative launch only with all of its CTAs resident
 * (work on other streams delays it rather than starving a barrier); if it
 * refuses the grid, or with on = 0, three launches per step run instead.
 * Both forms give the same results up to the order of floating-point sums.
 * hef_resistance_batched always uses the per-step form.  on = 2 exercises
 * the timeout path: the persistent form is launched (plainly) with twice the
 * CTAs that can be resident, so its first barrier cannot complete; the
 * launch ends after the wait limit with HEF_WAIT_TIMEOUT set and later calls
 * on that incidence do no work until it is rebuilt. */
hef_status hef_set_krylov_persistent(int32_t on);
/* Krylov basis with a tape for the backward: computes exactly what
 * hef_krylov_basis computes and also stores in `tape` (device, 256-byte
 * aligned, hef_krylov_tape_bytes bytes, caller-owned) what
 * hef_edge_resistance_backward reads: the recurrence coefficients and norms
 * of every chain and the chain vectors x_0 .. x_k of both expansions (in the
 * basis dtype).  The tape is (k + 1) * (2n + m) * S elements plus a few KB. */
size_t hef_krylov_tape_bytes(const hef_incidence* inc, int32_t k, int32_t S,
                             int32_t dtype);
hef_status hef_krylov_basis_tape(const hef_incidence* inc, int32_t k,
                                 int32_t S, int32_t dtype,
                                 const double* x0_clique,
                                 const double* x0_star, void* V, int64_t ldv,
                                 void* tape, size_t tape_bytes,
                                 void* workspace, size_t workspace_bytes,
                                 void* stream);
/* Krylov pool of one expansion, or both (ops = HEF_OPS_*).  HEF_OPS_STAR is
 * the star-only pool of the earlier HyperEF method, which Section III-A.3
 * contrasts with the mixed pool; HEF_OPS_BOTH is hef_krylov_basis.  With a
 * single expansion V gets K = k S columns, column (j-1) S + s holding the
 * j-th chain vector of start s, exactly the columns of that expansion in
 * hef_krylov_basis (k S <= 256 for a single expansion; ldv >= k S).  The
 * chains of both expansions are computed (the kernels fuse them) and the
 * other expansion's columns are discarded.  Workspace:
 * hef_krylov_ops_workspace_bytes. */
size_t hef_krylov_ops_workspace_bytes(const hef_incidence* inc, int32_t k,
                                      int32_t S, int32_t dtype, int32_t ops);
hef_status hef_krylov_basis_ops(const hef_incidence* inc, int32_t k,
                                int32_t S, int32_t dtype, int32_t ops,
                                const double* x0_clique,
                                const double* x0_star, void* V, int64_t ldv,
                                void* workspace, size_t workspace_bytes,
                                void* stream);
/* ------------------------------------------------------------------------
 * Orthonormalisation (Algorithm 1 step 4): in place, V (n x K, ldv, dtype)
 * becomes Q with orthonormal, mean-free columns spanning the mean-free parts
 * of V's columns, in column order (Q = (I - 11^T/n) V R^-1 with R upper
 * triangular, positive diagonal).  CholQR2: Gram matrix, FP64 Cholesky,
 * triangular apply, twice.  A column whose squared norm after removing the
 * mean and the earlier columns is <= tol * its squared norm as given (tol
 * 1e-12 for HEF_F64, 1e-5 for HEF_F32; a Cholesky pivot resolves relative
 * residual norms only down to about sqrt(machine epsilon)) is dropped: its Q
 * column is zero and scoring ignores it.
 * R_out (K x K double, row-major, nullable) receives R.  rank_out (one int32,
 * nullable) receives the number of kept columns.  K <= 512, n >= 1.
 * ---------------------------------------------------------------------- */
size_t hef_orthonormalize_workspace_bytes(int64_t n, int32_t K, int32_t dtype);

hef_status hef_orthonormalize(int64_t n, int32_t K, int32_t dtype, void* V,
                              int64_t ldv, double* R_out, int32_t* rank_out,
                              void* workspace, size_t workspace_bytes,
                              void* stream);

/* ------------------------------------------------------------------------
 * Edge resistance (Algorithm 1 steps 5 and 7; Eqs. non-linerQ, ratios, R).
 *
 * For basis column i of Q (n x K, ldq, dtype) and hyperedge e with >= 2
 * pins: spread_{e,i} = max_{p in e} Q[p,i] - min_{p in e} Q[p,i];
 * Q_H[i] = sum_e w_e spread_{e,i}^2 (FP64, fixed summation order);
 * r_{e,i} = spread_{e,i}^2 / Q_H[i] for columns with Q_H[i] > 1e-300;
 * R_e = max_i r_{e,i} (HEF_REDUCE_MAX) or sum_i r_{e,i} (HEF_REDUCE_SUM).
 * HEF_REDUCE_EMBED (a reading of "p and q are the most distant nodes in the
 * embedding space"): per hyperedge the pin pair (p, q) with the largest
 * squared Euclidean distance over all K columns (summed in ascending column
 * order in FP64; ties to the first pair in pin-position order), then
 * r_{e,i} = (Q[p,i] - Q[q,i])^2 / Q_H[i] in FP64, R_e = max_i (lowest i on
 * ties), pmax / pmin = p, q ordered by their values in column argvec (p
 * first when equal); Q_H is unchanged.  Work grows as |e|^2 K per hyperedge.
 * Precision: spreads in the basis dtype; the arg-max column is chosen on the
 * ratios in that dtype; R_e is formed in FP64 as spread^2 times the FP64
 * 1/Q_H (within an ulp or two of the quotient).  The workspace call and the
 * no-alloc call sum Q_H in the same order; the no-alloc call gathers Q again
 * instead of storing the spreads.
 * Outputs are indexed by the caller's hyperedge ids:
 *   R_out[m] double; QH_out[K] double (nullable);
 *   argvec[m] (nullable): the i attaining the max (lowest i on ties, -1 if
 *   none); pmax[m], pmin[m] (nullable): the vertices attaining the max and
 *   min of column argvec on e (lowest position within e on ties, -1 if none).
 * K <= 512.
 * ---------------------------------------------------------------------- */
size_t hef_edge_resistance_workspace_bytes(const hef_incidence* inc,
                                           int32_t K);

hef_status hef_edge_resistance(const hef_incidence* inc, const void* Q,
                               int64_t ldq, int32_t K, int32_t dtype,
                               int32_t reduce, double* R_out, double* QH_out,
                               int32_t* argvec, int32_t* pmax, int32_t* pmin,
                               void* workspace, size_t workspace_bytes,
                               void* stream);

/* ------------------------------------------------------------------------
 * Algorithm 1 end to end from HOST arrays (a service of the library for C
 * callers that hold the hypergraph in host memory): copies eptr[m+1],
 * pins[P], w[m], x0_clique[n x S], x0_star[(n+m) x S] (host; pinned memory
 * makes the copies asynchronous) into `workspace` (DEVICE, 256-byte aligned,
 * hef_resistance_host_workspace_bytes), runs hef_build_incidence,
 * hef_krylov_basis, hef_orthonormalize and hef_edge_resistance
 * (HEF_REDUCE_MAX) on `stream`, copies R (m doubles) to the host array
 * R_out and synchronises `stream`.  The start vectors are copied on a side
 * stream of the library (one per calling thread and device, created on the
 * first call) that waits for the work already queued on `stream` and joins
 * it before the Krylov stage, so that their copy overlaps the incidence
 * build.  Returns the first error of those calls,
 * HEF_ERR_INVALID_INPUT when the device-side validation failed, or
 * HEF_ERR_TIMEOUT when a bounded device wait expired.
 *
 * Repeated calls: when a thread calls again with the same host arrays,
 * workspace, sizes, form and stream as its previous call, and every host
 * array is page-locked, the second such call captures its device work (the
 * copies, the four calls, the copy of R) into a CUDA graph on a private
 * stream of the library, and later calls launch that graph on `stream`
 * instead of some forty separate launches.  The graph copies the host
 * arrays when it runs, so new contents in the same buffers are scored; it
 * keeps the Krylov launch form chosen when it was captured
 * (hef_set_krylov_persistent), and its launches do not pass through the
 * library's launch accounting (hef_launch_count, hef_trace_kernels).  A call
 * with anything different, or with pageable host arrays, runs as above.
 * ---------------------------------------------------------------------- */
size_t hef_resistance_host_workspace_bytes(int64_t n, int64_t m, int64_t P,
                                           int32_t k, int32_t S,
                                           int32_t dtype);
hef_status hef_resistance_host(int64_t n, int64_t m, int64_t P,
                               const int64_t* eptr, const int32_t* pins,
                               const double* w, const double* x0_clique,
                               const double* x0_star, int32_t k, int32_t S,
                               int32_t dtype, int32_t clique_mode,
                               double* R_out, void* workspace,
                               size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Backward of the whole path (Algorithm 1 steps 3-7).  The paper defines
 * only the forward; this is its derivative: given g = dL/dR (R as returned
 * by hef_edge_resistance with HEF_REDUCE_MAX), it writes
 *   dw[m]              dL/dw_e (caller's hyperedge order), through Q_H, the
 *                      expansion weights w/(|e|-1) (or w/C(|e|,2)) and w/|e|,
 *                      the degrees, and the degree-weighted deflation of the
 *                      starts;
 *   dx0_clique[n x S]  dL/d x0_clique (nullable);
 *   dx0_star[(n+m) x S] dL/d x0_star, same layout as x0_star (nullable).
 * The routing of the forward is held: the column argvec[e] and the pins
 * attaining the max and min of each column on e (lowest position on ties) do
 * not move under a small change of the inputs, so R is piecewise smooth and
 * this is the derivative of the smooth piece.  The Krylov recurrence
 * coefficients only change V by an upper-triangular factor, which Q does
 * not see, so they carry no gradient.
 * Inputs are the forward's, unchanged: x0_clique / x0_star as given to the
 * Krylov call; tape from hef_krylov_basis_tape with the same arguments, or
 * NULL to recompute it inside the workspace (query with recompute = 1); Q
 * (n x ldq, dtype) and R_fac (K x K, FP64) from hef_orthonormalize; QH,
 * argvec and R from hef_edge_resistance.  Columns dropped by the
 * orthonormalisation carry no gradient.  dR is device FP64 (m, caller
 * order).  The scoring adjoint is FP64; the orthonormalisation and
 * Krylov-chain adjoints run in the basis dtype (FP32 for HEF_F32) with FP64
 * partial sums and weight-gradient sums; the Q_H adjoint is summed with FP64
 * atomics, so two runs agree to rounding, not bit for bit.
 * ---------------------------------------------------------------------- */
/* Memory policy of the backward (no counterpart in the paper): whether the
 * forward should keep the Krylov tape for the backward (*use_tape = 1:
 * hef_krylov_basis_tape) or the backward should recompute the chains
 * (*use_tape = 0: hef_krylov_basis, then the backward with tape = NULL,
 * whose workspace holds the chains only while it runs).  The tape
 * (*tape_bytes, nullable; hef_krylov_tape_bytes) is kept when it fits
 * budget_bytes, or with budget_bytes = 0 half of the device memory that
 * cudaMemGetInfo reports free on the current device.  Synchronous query of
 * the device's memory; no device work. */
hef_status hef_backward_plan(const hef_incidence* inc, int32_t k, int32_t S,
                             int32_t dtype, uint64_t budget_bytes,
                             int32_t* use_tape, uint64_t* tape_bytes);
size_t hef_edge_resistance_backward_workspace_bytes(const hef_incidence* inc,
                                                    int32_t k, int32_t S,
                                                    int32_t dtype,
                                                    int32_t recompute);
hef_status hef_edge_resistance_backward(
    const hef_incidence* inc, int32_t k, int32_t S, int32_t dtype,
    const double* x0_clique, const double* x0_star, const void* tape,
    size_t tape_bytes, const void* Q, int64_t ldq, const double* R_fac,
    const double* QH, const int32_t* argvec, const double* R, const double* dR,
    double* dw, double* dx0_clique, double* dx0_star, void* workspace,
    size_t workspace_bytes, void* stream);
/* ------------------------------------------------------------------------
 * Batched form: Algorithm 1 on G independent hypergraphs of uneven sizes
 * (e.g. the levels of a multilevel hierarchy) in one call.  The paper scores
 * one hypergraph at a time; batching is a service of the library.
 *
 * `items` is a HOST array of G descriptors; every pointer inside is device
 * memory with the meaning of hef_build_incidence (eptr, pins, w), of
 * hef_krylov_basis (x0_clique, x0_star) and of hef_edge_resistance (R_out,
 * QH_out, argvec, pmax, pmin; all but R_out nullable).  status_out
 * (nullable, 2 words) receives the item's device status word and first bad
 * hyperedge (hef_incidence_check's detail and where), so a caller can check
 * every item after the stream has run.
 *
 * Each item runs the whole path (HEF_REDUCE_MAX) on one stream of a
 * per-device pool of 16 streams; chains of different items overlap.  The
 * Krylov stage (hef_set_batch_krylov_form): form 1 (default) runs the k
 * steps of every item in one cooperative launch (up to 64 items per
 * launch), each item on a share of the CTAs in proportion to its work
 * (at least one), with its own grid barriers and partial sums — between the
 * items' incidence builds and Krylov starts (on their streams) and their
 * CholQR2 and scoring (on their streams again); form 0 runs each item's
 * Krylov steps as per-step launches on its stream.  The call forks from `stream` with an event and joins back, so it
 * can be captured in a CUDA graph; the pool is created by the first call on
 * a device, which must happen outside stream capture.  schedule[g] (HOST,
 * nullable) is the pool stream of item g in [0, nstreams); NULL assigns items
 * longest first to the least loaded stream (hef_batch_schedule).  With form 0
 * the results are identical, bit for bit, to one hef_build_incidence /
 * hef_krylov_basis / hef_orthonormalize / hef_edge_resistance sequence per
 * item made with the per-step Krylov form (hef_set_krylov_persistent(0));
 * with form 1 they equal them up to the order of floating-point sums.
 * The pool and its fork/join events are shared by every batched call on a
 * device: make batched calls from one host thread at a time.
 * hef_batch_autotune waits for `stream`, then for both Krylov forms and
 * nstreams = 1, 2, 4, 8, 16 (each with its longest-first schedule) captures
 * the batch as a CUDA graph on a private stream and times three replays; it
 * returns the fastest: nstreams_out, schedule_out[G] (HOST), ms_out
 * (nullable, ms per batch), and leaves the calling thread set to the faster
 * Krylov form (hef_batch_krylov_form reads it).  It writes the items'
 * outputs while timing and must not be called inside a stream capture.
 * ---------------------------------------------------------------------- */
typedef struct hef_batch_item {
  int64_t n, m, P;
  const int64_t* eptr;
  const int32_t* pins;
  const double* w;
  const double* x0_clique;
  const double* x0_star;
  double* R_out;
  double* QH_out;
  int32_t* argvec;
  int32_t* pmax;
  int32_t* pmin;
  uint32_t* status_out;
} hef_batch_item;
size_t hef_batch_workspace_bytes(const hef_batch_item* items, int32_t G,
                                 int32_t k, int32_t S, int32_t dtype);
hef_status hef_batch_schedule(const hef_batch_item* items, int32_t G,
                              int32_t k, int32_t S, int32_t nstreams,
                              int32_t* schedule);
hef_status hef_resistance_batched(const hef_batch_item* items, int32_t G,
                                  int32_t k, int32_t S, int32_t dtype,
                                  int32_t clique_mode, const int32_t* schedule,
                                  int32_t nstreams, void* workspace,
                                  size_t workspace_bytes, void* stream);
/* Krylov stage of hef_resistance_batched for calls from this thread: 1 = one
 * cooperative launch for all items (default), 0 = per-step launches per item. */
hef_status hef_set_batch_krylov_form(int32_t form);
int32_t hef_batch_krylov_form(void);
hef_status hef_batch_autotune(const hef_batch_item* items, int32_t G,
                              int32_t k, int32_t S, int32_t dtype,
                              int32_t clique_mode, void* workspace,
                              size_t workspace_bytes, void* stream,
                              int32_t* nstreams_out, int32_t* schedule_out,
                              float* ms_out);
/* ------------------------------------------------------------------------
 * Consumers of the scores: Algorithm 1 step 6 and one coarsening level of
 * Algorithm 2 (Section III-B, steps 4-10) with Eq. R_W_update (Section
 * III-A.3, "Multilevel Effective Resistance Clustering").  The paper fixes
 * neither the threshold nor any tie rule; these calls implement the
 * following reading of it, and their results are a deterministic function
 * of the inputs (integer atomics only; FP64 sums in the stated orders with
 * round-to-nearest operations), equal bit for bit to a sequential CPU
 * statement of the same rules.
 *
 * hef_sort_resistance (Algorithm 1 step 6): order[m] = the hyperedge ids in
 * ascending R (finite), ties by ascending id.
 *
 * hef_coarsen_level, with the hyperedges as given to hef_build_incidence
 * (eptr[m+1], pins[P], w[m], caller order; `inc` is that incidence):
 *  1. Eq. R_W_update: R_upd[e] = (sum over e's pins, in pin order from 0.0,
 *     of eta[v]) + R[e]; eta (n, nullable = zeros) are the vertices'
 *     supernode weights from the previous level.
 *  2. order = hyperedges by ascending R_upd, ties by id.
 *  3. delta = the given delta (>= 0), or with delta < 0 the quantile-th
 *     quantile of R_upd over the hyperedges with >= 2 pins: the value at
 *     position floor(quantile (c - 1)) of their ascending order (c of them;
 *     +inf if c = 0).  *out->delta receives it.
 *  4. Greedy contraction in that order: a hyperedge with >= 2 pins and
 *     R_upd < delta is contracted when none of its pins belongs to a
 *     hyperedge contracted before it; owner[v] = the contracted hyperedge
 *     that v joined, -1 for isolated vertices.
 *  5. cluster[v]: a new id, in ascending vertex order, for every isolated
 *     vertex and for the smallest pin of every contracted hyperedge; the
 *     other pins take their supernode's id (nc ids).
 *  6. Local clustering (Section III-B.2; only when Q is given: Q n x ldq of
 *     dtype, K columns, QH[K] from hef_edge_resistance): every isolated
 *     vertex p joins the supernode c, among those of its co-pins (in the
 *     hyperedges containing p) formed by a contraction, that minimises
 *     d = max over i with QH[i] > 1e-300 of (Q[p,i] - mu_c[i])^2 / QH[i],
 *     mu_c = the mean Q row of c's members (summed in the forming
 *     hyperedge's pin order); ties to the smallest c.  target[p] = c (an id
 *     of step 5) or -1, dist[p] = d (0 if none).
 *  7. Weights: a supernode's weight is the R_upd of its hyperedge, an
 *     isolated vertex keeps eta[v]; each joining seed p adds (eta[p] +
 *     dist[p]) to its supernode's weight, in ascending p.
 *  8. final_cluster[v]: compact ids (nf of them) in the order of each
 *     cluster's smallest vertex; eta_out[nf] their weights (the next level's
 *     eta).
 *  9. Coarse hypergraph (Algorithm 2 step 6): each hyperedge's pins mapped
 *     to final ids, the first occurrence of each id kept in pin order;
 *     hyperedges left with < 2 pins are dropped, the rest keep their weight
 *     and relative order: ceptr[m'+1] (int64), cpins[P'], cw[m'], emap[m']
 *     (the hyperedge it came from).
 * counts[5] = {nc, nf, m', P', status}; status is nonzero when a bounded
 * grid-wide wait of the contraction ran out (results then invalid).  The
 * contraction is one cooperative launch (rounds of a fixed point that equals
 * the sequential greedy rule).  All outputs are caller-owned device arrays
 * sized for the fine hypergraph: R_upd, order, cw, emap [m]; ceptr [m+1];
 * cpins [P]; owner, cluster, target, final_cluster [n]; dist, eta_out [n];
 * delta [1]; counts [5].  Workspace: hef_level_workspace_bytes(n, m, K)
 * (K = 0 without Q); hef_sort_resistance needs hef_level_workspace_bytes(0,
 * m, 0).
 * ---------------------------------------------------------------------- */
typedef struct hef_level_out {
  double* R_upd;
  int32_t* order;
  double* delta;
  int32_t* owner;
  int32_t* cluster;
  int32_t* target;
  double* dist;
  int32_t* final_cluster;
  double* eta_out;
  int32_t* counts;
  int64_t* ceptr;
  int32_t* cpins;
  double* cw;
  int32_t* emap;
} hef_level_out;

size_t hef_level_workspace_bytes(int64_t n, int64_t m, int32_t K);
hef_status hef_sort_resistance(int64_t m, const double* R, int32_t* order,
                               void* workspace, size_t workspace_bytes,
                               void* stream);
/* `out` is a HOST struct of device pointers. */
hef_status hef_coarsen_level(const hef_incidence* inc, const int64_t* eptr,
                             const int32_t* pins, const double* w,
                             const double* R, const double* eta,
                             const void* Q, int64_t ldq, int32_t K,
                             int32_t dtype, const double* QH, double delta,
                             double quantile, const hef_level_out* out,
                             void* workspace, size_t workspace_bytes,
                             void* stream);

/* ------------------------------------------------------------------------
 * Edge resistance without caller-provided device memory.  The paper has no
 * counterpart: this is a service of the library.
 *
 * Some callers cannot give the library a workspace: plain C code that only
 * holds the pointers it was handed and has no device allocator of its own, or
 * a host application whose memory pool already owns all of the GPU's free
 * memory (cudaMalloc would fail, and it also synchronises the device, which a
 * latency-critical caller must not do in mid-stream).  This call computes
 * exactly what hef_edge_resistance computes and allocates nothing: its
 * scratch (per-CTA partial sums of Q_H, Q_H and 1/Q_H, a completion counter)
 * is a fixed 2 MiB array compiled into the library, which every GPU that
 * loads the library reserves until the process exits.
 *  - The caller still provides Q and the outputs (same meaning as
 *    hef_edge_resistance); K must be <= 512 (HEF_ERR_UNSUPPORTED otherwise).
 *  - The first call on a device looks up the array's device address (with
 *    that device current) and caches it; make that first call before any
 *    stream capture.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind.  Calls ordered on one stream are safe; calls that overlap on the
 *    GPU (different streams or host threads without ordering) race on it.
 * ---------------------------------------------------------------------- */
hef_status hef_edge_resistance_noalloc(const hef_incidence* inc,
                                       const void* Q, int64_t ldq, int32_t K,
                                       int32_t dtype, int32_t reduce,
                                       double* R_out, double* QH_out,
                                       int32_t* argvec, int32_t* pmax,
                                       int32_t* pmin, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HEF_H_ */
