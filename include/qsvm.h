/*
 * qsvm.h -- C ABI of libqsvm: GB300-native quantum-kernel estimation for QSVMs
 * (after arXiv 2405.02630, "Validating Large-Scale Quantum Machine Learning:
 * Efficient Simulation of Quantum Support Vector Machines Using Tensor Networks").
 *
 * The library computes quantum-kernel matrices
 *     K(x_i, x_j) = |<psi(x_j)|psi(x_i)>|^2 = |<0^n| U^dagger(x_j) U(x_i) |0^n>|^2
 * (Sec. 2, Eq. 3 and Eq. 4) for the n-qubit linear-chain feature map of Sec. 3.2
 * (CNOTs in a linear topology, one qubit per feature).  One repetition of U(x):
 * H on every qubit; RZ(2 x_k) on every qubit; then for k = 0..n-2 the block
 * CNOT(k,k+1) . RZ_{k+1}(2 (pi - x_k)(pi - x_{k+1})) . CNOT(k,k+1).
 * RZ(theta) = diag(exp(-i theta/2), exp(+i theta/2)).  reps repetitions.
 *
 * Each state U(x)|0^n> is built exactly (no truncation) as a matrix product
 * state of bond dimension chi = 2^reps, and every kernel entry is the overlap of
 * two such states contracted along the chain (the tensor-network kernel of
 * Algorithm 2, with the chain's fixed left-to-right contraction order).
 *
 * Conventions shared by every entry point
 *   - Pointers named X, mps, K, logK are DEVICE pointers owned by the caller
 *     (e.g. allocated through PyTorch); the library never allocates, frees or
 *     retains them.  Buffers handed to the library must be 16-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls only enqueue work on it and return; they never synchronise, except
 *     qsvm_device_status(), which says so.
 *   - Return value: QSVM_OK (0) or a negative qsvm_status.  Argument errors are
 *     detected on the host before anything is enqueued.  qsvm_last_error()
 *     returns a thread-local message for the last failing call on this thread.
 *   - Kernels never trap.  A wait inside a kernel that exceeds its bound makes
 *     the kernel record QSVM_ERR_TIMEOUT in a device status word and return;
 *     qsvm_device_status() reads it.
 *   - All indices are 64-bit; matrices are row-major with explicit leading
 *     dimensions (in elements).
 */
#ifndef QSVM_H
#define QSVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum qsvm_status {
  QSVM_OK = 0,
  QSVM_ERR_ARG = -1,            /* bad pointer, size, alignment or leading dim  */
  QSVM_ERR_CHI = -2,            /* reps outside 1..3 (chi = 2^reps > 8)          */
  QSVM_ERR_CUDA = -3,           /* a CUDA runtime call or launch failed          */
  QSVM_ERR_TIMEOUT = -4,        /* a bounded in-kernel wait ran out              */
  QSVM_ERR_UNIMPLEMENTED = -5,  /* valid request this build does not provide     */
  QSVM_ERR_WORKSPACE = -6       /* caller workspace smaller than required        */
};

/* ---- arithmetic of the pair contraction --------------------------------- */
enum qsvm_precision {
  /* FP64 everywhere: the parity path. */
  QSVM_FP64 = 0,
  /* Plain FP32 site tensors and FP32 environment on the CUDA cores; exact
   * power-of-two renormalisation.  Fastest; relative error grows with n. */
  QSVM_FP32 = 1,
  /* Split FP32: every site tensor and environment entry is hi + lo, with hi on a
   * fixed binary grid so that hi*hi products and their short sums are exact in
   * FP32 FMAs, and the lo terms carried as FP32 corrections.  Accuracy near
   * FP64 (|dK| ~ 1e-8 at n = 784) at FP32-pipe speed. */
  QSVM_FP32_SPLIT = 2
  /* There is no tensor-core value.  TF32 operands (|dK| ~ 0.25 at n = 784) and
   * two-term BF16 operands (~3e-3) miss the 1e-6 bar outright (CPU emulation of
   * the arithmetic).  Three-term TF32 operands with FP32 accumulation would meet
   * it, but the only products with an operand shared across pairs are 2 x 2
   * complex (one m16n8k4 MMA per 4 pairs) and the pairs must be regrouped through
   * shared memory twice per site: on GB300 a kernel doing only those MMAs, the
   * operand re-splits and the regrouping ran at 4.2e7 entries/s at n = 784,
   * reps = 2, against 8.0e7 for the complete QSVM_FP32_SPLIT contraction. */
};

/* ---- MPS storage ---------------------------------------------------------
 * Records per (point, site), point-major: record (i, k) of an array at byte
 * i * qsvm_mps_point_bytes(...) + k * qsvm_mps_record_bytes(reps, precision)
 * (k = 0 .. n_qubits - 1, and k = n_qubits for the virtual site of the gauged
 * form).  With
 * P = exp(-i x_k), T = exp(-i theta_{k-1}), theta_{k-1} = (pi - x_{k-1})(pi - x_k)
 * (T = 1 at site 0), z(b) = 1 - 2b, right bond index u = 2p + s and left bond
 * index t = 2q + c, the site tensor is A_k[sigma][t][u] = 0 unless sigma == s
 * (the last layer is diagonal), and its blocks a_cs[q][p] = A_k[s][2q+c][2p+s]
 * satisfy a_1s = r_s a_0s with r_0 = conj(T^2) and r_1 = T^2.
 *
 * Phase form (reps = 2, QSVM_FP32): every entry is +-1/2 times 1, T^2, P^2 or
 * P^2 T^2 or a conjugate, a_00 = (1/2) [[P^2 T^2, 1], [P^2, T^2]] and
 * a_01 = (1/2) [[1, -conj(P^2 T^2)], [conj(T^2), -conj(P^2)]] (rows q, columns p),
 * and the record holds the three phases V0 = T^2, V1 = P^2, V2 = P^2 T^2, per
 * value its a-form then its b-form entry (below), 96 bytes.  The last site's
 * tensor keeps its right bond open (its layer-1 spin is summed by the
 * contraction).  One array of records.
 *
 * Gauged form (reps = 2, QSVM_FP64 and QSVM_FP32_SPLIT): after the diagonal change of bond
 * basis that makes row t = 0 of every site tensor one, both blocks of site k are
 * [[1, 1], [alpha_k, beta_k]] with alpha_k = conj(V2^{k-1} V0^k) and
 * beta_k = conj(V2^{k-1}) V0^k (V^k the phases of site k, V2^{-1} = 1), and
 * a_1s = r'_s diag(1, -1) a_0s with r'_0 = alpha_k, r'_1 = beta_k.  A virtual
 * site n with alpha_n = beta_n = conj(V2^{n-1}) undoes the basis change on the
 * last bond.  QSVM_FP64: a record holds alpha then beta as (re, im) doubles, 32
 * bytes, n_qubits + 1 records per point in one array.  QSVM_FP32_SPLIT: a record
 * holds alpha then beta, each as its hi entry (re and im on the 2^-11 grid) then
 * its lo entry, 64 bytes; a buffer holds n_qubits + 1 records per point in two
 * arrays: the row-side a-forms, then the column-side b-forms.
 *
 * Split FP32 at reps = 3: the gauged records of reps = 2 (the same alpha, beta and
 * virtual site, 64 bytes per record, two arrays of n_qubits + 1 records per point).
 * The same change of bond basis makes both blocks of a chi = 8 site the signed
 * Kronecker square (-1)^{q1 q2} M[q1][p1] M[q2][p2] of M = [[1, 1], [alpha_k, beta_k]]
 * (q = q1 + 2 q2, p = p1 + 2 p2, q1 the first layer) and the c = 1 rows
 * r'_s diag(1, 1, -1, -1) times the c = 0 rows.
 *
 * Block form (reps = 1; reps = 3 in FP64 and FP32): the record stores the two chi/2 x chi/2 blocks
 * a_00, a_01, each row-major over (q, p), then the phase r_0, 16 bytes per value:
 *   QSVM_FP64        (re, im) as two doubles;
 *   QSVM_FP32        one "form" entry of four floats;
 *   QSVM_FP32_SPLIT  per block: the chi^2/4 "hi" form entries (re and im on the
 *                    2^-11 grid), then the chi^2/4 "lo" form entries; the phase
 *                    as a hi entry then a lo entry.
 * Site 0 has a left bond of dimension 1 (only t = 0 is nonzero); the last site
 * has a right bond of dimension 2 holding the physical index (u = sigma, p = 0).
 * The FP32 block formats hold two arrays of records: first the row-side a-forms,
 * then the column-side b-forms.
 *
 * Forms: an a-form entry of a complex value A is (re, im, -im, re) = (A, iA);
 * a b-form entry is (re, -im, im, re) = (conj A, i conj A).  With them a complex
 * multiply-add is two packed FP32x2 FMAs with one broadcast operand.
 * qsvm_mps_point_bytes() is the size of one point's records in one array (the
 * row stride of an array): mps + m * qsvm_mps_point_bytes(...) passed as mps_a of
 * qsvm_kernel_cross addresses the points from m on of a buffer (mps_a is read
 * through its row-side array only).  qsvm_mps_bytes() is the size of a whole
 * buffer; both return 0 for arguments outside their range.  The layout is
 * private to this library: produce it with qsvm_build_mps. */
size_t qsvm_mps_record_bytes(int32_t reps, int32_t precision);
size_t qsvm_mps_point_bytes(int32_t n_qubits, int32_t reps, int32_t precision);
size_t qsvm_mps_bytes(int32_t n_qubits, int32_t reps, int64_t n_points, int32_t precision);

/* qsvm_build_mps -- exact MPS of U(x)|0^n> for every row of X (Sec. 3.2 circuit;
 * the state whose overlaps Eq. 4 needs).
 *   X          device, n_points x n_qubits float64, row-major (features = angles,
 *              already scaled as the caller wants; the paper uses PCA-reduced,
 *              scaled pixels, Sec. 3.2).
 *   precision  storage format of the output records (the build itself is FP64).
 *   mps        device output, at least qsvm_mps_bytes(...) bytes (mps_bytes).
 * In FP64, site by site.  reps = 1, 3: gate by gate (H and RZ act on the physical
 * index; the commuting CNOT.RZ.CNOT blocks of one repetition act as a bond-2
 * diagonal MPO that copies each spin onto the bond and applies
 * exp(-i theta Z_k Z_{k+1}), theta = (pi - x_k)(pi - x_{k+1}), on the right-hand
 * site).  reps = 2: the same gates applied to the rows t = 0, 2 (right bond open),
 * and the three phases read off three of the resulting entries (split FP32:
 * alpha and beta formed from the phases of sites k - 1 and k).
 * Errors: QSVM_ERR_ARG (null, n_qubits < 2, n_points < 1, mps_bytes too small,
 * misaligned), QSVM_ERR_CHI (reps outside 1..3), QSVM_ERR_CUDA. */
int32_t qsvm_build_mps(const double* X, int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                       void* mps, size_t mps_bytes, void* stream);

/* qsvm_kernel_gram -- symmetric train x train kernel matrix (Algorithm 2 with
 * its symmetrisation step): K[i*ldk + j] = |<psi_j|psi_i>|^2 for all i, j.
 * Only pairs i <= j are contracted (the diagonal too, it is computed rather
 * than set to 1) and K[j][i] is written as a bit-exact copy of K[i][j].
 *   mps   device, built by qsvm_build_mps with the same n_qubits, reps, precision.
 *   K     device float64, n_points rows, ldk >= n_points.
 *   logK  device float64 or NULL; if given, ln K (-inf where the amplitude is 0);
 *         ldl >= n_points.  K underflows to 0 below ~1e-308 while logK stays exact.
 * No workspace: each pair's environment lives in registers (or, at reps = 3 in
 * split FP32, in the CTA's shared memory) for the whole chain, and tiles write
 * their results straight into K, so the call takes no scratch argument.
 * Errors: QSVM_ERR_ARG, QSVM_ERR_CHI, QSVM_ERR_CUDA. */
int32_t qsvm_kernel_gram(const void* mps, int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                         double* K, int64_t ldk, double* logK, int64_t ldl, void* stream);

/* qsvm_kernel_cross -- test x train kernel (Algorithms 1-3 with datasize1 !=
 * datasize2; never symmetrised): K[i*ldk + j] = |<psi(train_j)|psi(test_i)>|^2.
 *   mps_a  device MPS of the n_a test points; mps_b of the n_b train points.
 *   K      device float64, n_a rows, ldk >= n_b; logK as above (ldl >= n_b).
 * Errors: as qsvm_kernel_gram. */
int32_t qsvm_kernel_cross(const void* mps_a, int64_t n_a, const void* mps_b, int64_t n_b, int32_t n_qubits,
                          int32_t reps, int32_t precision, double* K, int64_t ldk, double* logK, int64_t ldl,
                          void* stream);

/* qsvm_gram_host -- the symmetric Gram of host data, end to end: X (HOST,
 * n_points x n_qubits float64, row-major) is copied to the device, its MPS built
 * and its Gram computed, and K (HOST float64, ldk >= n_points) and, if logK
 * (HOST or NULL, ldl >= n_points) is given, ln K are copied back.  Page-locked
 * host memory lets the copies run asynchronously; pageable memory works but the
 * copies then synchronise with the host.  The Gram runs in up to eight launches of
 * whole tile bands (one for small problems: each launch gets at least four tiles
 * per SM), alternating between `stream` and a second compute stream (they
 * write disjoint tiles); once launches 0..c have completed, the rows of launch c
 * are final (a band's rows receive mirror writes only from earlier bands) and a
 * copy stream takes them to the host while later launches compute.
 *   ws     device scratch of qsvm_gram_host_workspace_bytes(n_points, n_qubits,
 *          reps, precision, logK != NULL) bytes, 256-byte aligned, owned by the
 *          caller: X, the MPS and K (and logK) are staged there.
 * Stream-ordered on `stream` (the helper streams are joined back into it): K and logK
 * are complete once `stream` has reached this point; the call itself does not
 * wait.  The helper streams are created and released by each call, so the call is
 * not meant for CUDA-graph capture (capture qsvm_build_mps + qsvm_kernel_gram on
 * device buffers instead), and one ws serves one call at a time.  Results are
 * bit-identical to qsvm_build_mps + qsvm_kernel_gram.
 * Errors: as qsvm_kernel_gram, and QSVM_ERR_ARG for a missing or short ws. */
size_t qsvm_gram_host_workspace_bytes(int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                                      int32_t with_logk);
int32_t qsvm_gram_host(const double* X, int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                       double* K, int64_t ldk, double* logK, int64_t ldl, void* ws, size_t ws_bytes, void* stream);

/* qsvm_cross_host -- the test x train kernel of host data, end to end: X_a (HOST,
 * n_a x n_qubits float64, the test points) and X_b (HOST, n_b x n_qubits, the train
 * points) are copied to the device and their MPS built; the kernel (K[i*ldk + j] as in
 * qsvm_kernel_cross, HOST float64, ldk >= n_b; logK HOST or NULL, ldl >= n_b) runs in
 * up to eight launches of whole tile rows (one for small problems: each launch gets at
 * least four tiles per SM), alternating between `stream` and a second compute stream,
 * and each launch's rows are copied to the host on a third stream while later
 * launches compute.
 *   ws  device scratch of qsvm_cross_host_workspace_bytes(n_a, n_b, n_qubits, reps,
 *       precision, logK != NULL) bytes, 256-byte aligned, owned by the caller.
 * Stream-ordered on `stream` as qsvm_gram_host (the same capture and workspace
 * caveats).  Results are bit-identical to qsvm_build_mps + qsvm_kernel_cross.
 * Errors: as qsvm_kernel_cross, and QSVM_ERR_ARG for a missing or short ws. */
size_t qsvm_cross_host_workspace_bytes(int64_t n_a, int64_t n_b, int32_t n_qubits, int32_t reps, int32_t precision,
                                       int32_t with_logk);
int32_t qsvm_cross_host(const double* X_a, int64_t n_a, const double* X_b, int64_t n_b, int32_t n_qubits,
                        int32_t reps, int32_t precision, double* K, int64_t ldk, double* logK, int64_t ldl, void* ws,
                        size_t ws_bytes, void* stream);

/* ---- sharding the symmetric Gram over independent workers ----------------
 * The upper-triangle pair tiles of a Gram are independent (Sec. 5: pairs are
 * distributed evenly over GPUs and the results gathered).  A tile is a
 * qsvm_gram_tile_dim() x qsvm_gram_tile_dim() block of pairs; with
 * T = ceil(n_points / tile_dim), tiles (ti, tj), ti <= tj, are numbered in bands
 * of 8 tile rows, within a band column by column, within a column row by row
 * (the order the kernels visit them in; qsvm_gram_tile_coords decodes one,
 * qsvm_gram_tile_list the range [tile_begin, tile_end) into host arrays ti, tj of
 * tile_end - tile_begin entries each, owned by the caller; QSVM_ERR_ARG for a range
 * outside [0, tiles], no tiles at all, or null arrays with a non-empty range).
 * qsvm_gram_partition splits [0, tiles) into `world` contiguous ranges of
 * near-equal pair count; qsvm_kernel_gram_tiles computes one range (writing both
 * K[i][j] and its mirror for every pair in it).  All but qsvm_kernel_gram_tiles
 * are pure host functions. */
int32_t qsvm_gram_tile_dim(int32_t reps, int32_t precision);
int64_t qsvm_gram_num_tiles(int64_t n_points, int32_t reps, int32_t precision);
int32_t qsvm_gram_partition(int64_t n_points, int32_t reps, int32_t precision, int32_t world, int32_t rank,
                            int64_t* tile_begin, int64_t* tile_end);
int32_t qsvm_gram_tile_coords(int64_t n_points, int32_t reps, int32_t precision, int64_t tile, int64_t* ti,
                              int64_t* tj);
int32_t qsvm_gram_tile_list(int64_t n_points, int32_t reps, int32_t precision, int64_t tile_begin,
                            int64_t tile_end, int64_t* ti, int64_t* tj);
int32_t qsvm_kernel_gram_tiles(const void* mps, int64_t n_points, int32_t n_qubits, int32_t reps,
                               int32_t precision, int64_t tile_begin, int64_t tile_end, double* K, int64_t ldk,
                               double* logK, int64_t ldl, void* stream);

/* ---- many Gram jobs in one persistent launch -------------------------------
 * Sec. 4.1 reuses one contraction path across all pairs and runs contractions
 * concurrently; here jobs of uneven qubit count and point count share one
 * persistent kernel: every CTA pulls the next pair tile from a device work
 * queue (jobs ordered by qubit count, largest first) until it is empty.
 * All jobs of one call share reps and precision. */
typedef struct qsvm_job {
  const void* mps;    /* device MPS of the job's points (qsvm_build_mps)            */
  int64_t n_points;
  int32_t n_qubits;   /* >= 2                                                      */
  int32_t reserved;   /* must be 0                                                 */
  double* K;          /* device, n_points x n_points, row-major, leading dim ldk    */
  int64_t ldk;
  double* logK;       /* device or NULL                                            */
  int64_t ldl;
} qsvm_job;

/* Device scratch the batch needs: the job table and the work-queue head. */
size_t qsvm_batch_workspace_bytes(int32_t n_jobs);

/* qsvm_kernel_batch -- every job's symmetric Gram (as qsvm_kernel_gram) in one
 * persistent launch.  jobs is a HOST array; ws is device scratch of at least
 * qsvm_batch_workspace_bytes(n_jobs) bytes (256-byte aligned) that must not be
 * used by anything else until the launch has finished on `stream`.  The job table
 * is copied into ws on `stream`.  Errors: QSVM_ERR_ARG, QSVM_ERR_CHI,
 * QSVM_ERR_WORKSPACE, QSVM_ERR_CUDA. */
int32_t qsvm_kernel_batch(const qsvm_job* jobs, int32_t n_jobs, int32_t reps, int32_t precision, void* ws,
                          size_t ws_bytes, void* stream);

/* A batch plan records the queue reset and the persistent launch in a CUDA graph
 * once (the job table is uploaded at creation) and replays it with one call.
 * The plan keeps using ws and the jobs' buffers until it is destroyed. */
typedef struct qsvm_batch_plan qsvm_batch_plan;
int32_t qsvm_batch_plan_create(const qsvm_job* jobs, int32_t n_jobs, int32_t reps, int32_t precision, void* ws,
                               size_t ws_bytes, qsvm_batch_plan** plan_out);
int32_t qsvm_batch_plan_launch(qsvm_batch_plan* plan, void* stream);
int32_t qsvm_batch_plan_destroy(qsvm_batch_plan* plan);

/* qsvm_kernel_batch_noalloc -- qsvm_kernel_batch without a workspace argument,
 * for callers that cannot allocate device memory (for example latency-bound
 * serving loops that must avoid cudaMalloc's device-wide synchronisation, or
 * hosts whose framework allocator already owns all device memory).  The paper has no
 * counterpart: this is an interface for such callers.  The job table and the
 * work-queue head live in a fixed 76 KiB array inside the library's device
 * image, present on every GPU that loads the library until the process exits;
 * at most 1024 jobs per call (more returns QSVM_ERR_WORKSPACE).  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Every call reuses the same
 * array and rewrites it (the queue head restarts at zero each call), so calls
 * whose work overlaps on the GPU race: order them on one stream or with events.
 * No device memory is allocated or freed.  Errors: as qsvm_kernel_batch. */
int32_t qsvm_kernel_batch_noalloc(const qsvm_job* jobs, int32_t n_jobs, int32_t reps, int32_t precision,
                                  void* stream);

/* ---- pipeline configurations and the autotuner ----------------------------
 * The pair kernels stream site records through shared memory in chunks; a
 * configuration fixes the bytes per point and chunk, the stages in flight, and
 * whether a CTA contracts a whole tile of pairs or a quarter of one.
 * Results are bit-identical for every configuration (the arithmetic and its
 * order do not depend on it); only speed differs.  The selection is per
 * (reps, precision), process-wide, and used by every later launch. */
int32_t qsvm_num_configs(void);
/* sites per chunk and stages of configuration `index` for (reps, precision) */
int32_t qsvm_config_info(int32_t index, int32_t reps, int32_t precision, int32_t* sites_per_chunk,
                         int32_t* stages);
/* qsvm_config_tile -- the block of pairs one CTA contracts under configuration
 * `index` (-1: the default) for (reps, precision): *pairs_per_side x *pairs_per_side
 * pairs with *threads_per_pair threads each (either output nullable).  The first
 * qsvm_num_configs()/2 configurations give each CTA a whole tile of
 * qsvm_gram_tile_dim() pairs per side, the others a quarter of one; tile indices,
 * partitions and tile lists are the same for both (they count whole tiles), and
 * the batch launches always use whole tiles.  Errors: QSVM_ERR_ARG for an index
 * out of range, QSVM_ERR_CHI for reps outside 1..3. */
int32_t qsvm_config_tile(int32_t index, int32_t reps, int32_t precision, int32_t* pairs_per_side,
                         int32_t* threads_per_pair);
int32_t qsvm_set_config(int32_t reps, int32_t precision, int32_t index); /* index -1: default */
int32_t qsvm_get_config(int32_t reps, int32_t precision);
/* qsvm_autotune -- times the Gram of `mps` (n_points, n_qubits) under every
 * configuration with CUDA events on `stream` (writing K as scratch), selects the
 * fastest for (reps, precision) and returns its index in *best_out; ms_out
 * (nullable, qsvm_num_configs() floats) gets each time (negative: not runnable).
 * Synchronises `stream`. */
int32_t qsvm_autotune(const void* mps, int64_t n_points, int32_t n_qubits, int32_t reps, int32_t precision,
                      double* K, int64_t ldk, void* stream, int32_t* best_out, float* ms_out);

/* ---- state-vector validator (small n) --------------------------------------
 * The state-vector recipe of Algorithm 1 on the GPU: every point's circuit is
 * simulated gate by gate (literal H, RZ, CNOT) on its 2^n complex128 amplitudes,
 * then K[i][j] = |<psi_j|psi_i>|^2 (Eq. 3-4) is formed from inner products over
 * the amplitudes in FP64.  It shares no code with the MPS builder or the pair
 * kernels, so it cross-checks them; cost grows as 2^n (n_qubits <= 24).
 *   X    device, n_points x n_qubits float64;  K device, n_points rows, ldk >= n_points
 *        (symmetric, diagonal computed);  ws device scratch of at least
 *        qsvm_sv_workspace_bytes() bytes (the state vectors).  reps is 1..64.
 * Errors: QSVM_ERR_ARG, QSVM_ERR_WORKSPACE, QSVM_ERR_CUDA. */
size_t qsvm_sv_workspace_bytes(int64_t n_points, int32_t n_qubits);
int32_t qsvm_sv_gram(const double* X, int64_t n_points, int32_t n_qubits, int32_t reps, double* K, int64_t ldk,
                     void* ws, size_t ws_bytes, void* stream);

/* ---- the support vector classifier on the kernel -----------------------------
 * Sec. 3.2 / Sec. 4.2 hand the quantum kernel matrix to an SVC (primal Eq. 1-2,
 * solved in its dual with the kernel in place of the inner product).  A binary
 * problem selects its n training points from a symmetric kernel matrix K by idx
 * and carries labels y = +1 / -1; qsvm_svc_fit solves the C-SVC dual
 *   min 1/2 a^T Q a - 1^T a,  Q_ij = y_i y_j K[idx_i][idx_j],  0 <= a <= C,  y^T a = 0
 * by sequential minimal optimisation with the maximal violating pair, stopping
 * when the optimality gap is below tol or after max_iter steps; one CTA per
 * problem, so all one-vs-one pairs of a multiclass fit share a launch.
 * b_out[p] (device) gets the bias and iters_out[p] (device) the steps taken.
 * qsvm_svc_decision writes F[r * n_problems + p] = sum_i a_i y_i Kx[r][idx_i] + b[p]
 * for m rows of a test x train kernel Kx.  ws: device scratch (256-byte aligned)
 * of qsvm_svc_workspace_bytes(problems) bytes (problem table and gradients). */
typedef struct qsvm_svc_problem {
  const int64_t* idx;  /* device, n row indices into K                            */
  const int8_t* y;     /* device, n labels +1 / -1                                */
  int64_t n;           /* >= 2                                                   */
  double* alpha;       /* device output, n dual coefficients                     */
} qsvm_svc_problem;
size_t qsvm_svc_workspace_bytes(const qsvm_svc_problem* problems, int32_t n_problems);
int32_t qsvm_svc_fit(const double* K, int64_t ldk, const qsvm_svc_problem* problems, int32_t n_problems, double C,
                     double tol, int64_t max_iter, double* b_out, int64_t* iters_out, void* ws, size_t ws_bytes,
                     void* stream);
int32_t qsvm_svc_decision(const double* Kx, int64_t ldk, int64_t m, const qsvm_svc_problem* problems,
                          int32_t n_problems, const double* b, double* F, void* ws, size_t ws_bytes, void* stream);

/* ---- diagnostics --------------------------------------------------------- */
/* Reads (and, if clear != 0, resets) the device status words written by this
 * library's kernels on the current device: QSVM_OK or QSVM_ERR_TIMEOUT.
 * Synchronises `stream`.  Returns QSVM_OK or QSVM_ERR_CUDA. */
int32_t qsvm_device_status(void* stream, int32_t clear, int32_t* status_out);
/* Exercises the failure path without a fault: launches one CTA that waits on an
 * mbarrier phase nothing completes, bounded by limit_ns (1e3 .. 2e9); the wait
 * gives up, the kernel records QSVM_ERR_TIMEOUT in the status word (read it with
 * qsvm_device_status) and returns, leaving the context usable. */
int32_t qsvm_selftest_wait_timeout(int64_t limit_ns, void* stream);
const char* qsvm_last_error(void);
const char* qsvm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QSVM_H */
