/*
 * tn.h -- C ABI of the tropical tensor-network contraction library (libtn.so).
 *
 * The library contracts the tensor network of a spin glass over the tropical
 * (max, +) semiring of Eq. 2 on one GB300 GPU (sm_103a) along a precomputed
 * pairwise contraction order.  Each pairwise step is a tensor transpose
 * followed by a batched max-plus GEMM (or a strided small-operand "gate"
 * contraction that needs no transpose); the same steps run over the counting
 * tuples (x, n) of Sec. II, with n kept modulo several 61-bit primes and
 * recovered exactly by the Chinese remainder theorem.  A backward traceback
 * through the contraction tree, recomputing intermediates from checkpoints,
 * yields the ground-state configuration (Sec. III).
 *
 * Conventions shared by every entry point
 *   - Spins are 0-based.  Ising (q = 2): state index 0 <-> sigma = +1,
 *     1 <-> sigma = -1, so the bond tensor is [[J, -J], [-J, J]] (Sec. II).
 *     Energy, Eq. 1: E = -sum_e J_e s_u s_v - sum_i h_i s_i.
 *     Potts (q = 3): E = -sum_e J_e delta(s_u, s_v); fields must be NULL.
 *   - Tensor elements hold negative energies, so the contracted scalar is
 *     V = max_sigma(-E) and E_min = -V (Sec. II).
 *   - All pointers are plain host pointers unless an argument says "device".
 *     Input arrays are copied; the caller keeps ownership of everything it
 *     passes.  Outputs go to caller-allocated buffers.
 *   - Device memory is owned by the context (one arena sized by the plan).
 *   - No C++ exception crosses this boundary: every call returns a status;
 *     tn_last_error() gives a one-line reason for the last failure.
 *   - A context is not thread-safe; use one context per host thread.
 *   - There is no CPU fallback: without a usable CUDA device the calls that
 *     compute return TN_ECUDA.
 */
#ifndef TN_H
#define TN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tn_ctx tn_ctx;

typedef enum {
  TN_OK = 0,
  TN_EINVAL = 1,     /* bad argument (sizes, ids, missing order, ...)      */
  TN_ENOMEM = 2,     /* plan does not fit the device budget / malloc fails */
  TN_ECUDA = 3,      /* a CUDA call failed, or no device                   */
  TN_ETIMEOUT = 4,   /* a bounded device-side wait gave up                 */
  TN_EOVERFLOW = 5,  /* count exceeds what the chosen primes can hold      */
  TN_ESTATE = 6      /* call out of order (e.g. tn_energy before tn_order) */
} tn_status;

/* ---- tn_build flags ---------------------------------------------------- */
#define TN_DTYPE_AUTO 0u   /* INT32 when every J and h is an integer, else FP32 */
#define TN_DTYPE_I32 1u    /* force INT32 (J, h must be integers, |.| < 2^20)   */
#define TN_DTYPE_F32 2u    /* force FP32                                         */
#define TN_DTYPE_MASK 3u

/* ---- tn_order methods --------------------------------------------------- */
#define TN_ORDER_SWEEP 0   /* seq = spin elimination sequence (e.g. row by row)  */
#define TN_ORDER_GREEDY 1  /* randomized greedy pair selection, best of restarts */
#define TN_ORDER_TREE 2    /* seq = explicit pairwise tree, 2 ids per step       */

/*
 * tn_build -- describe one spin-glass instance (Eq. 1 / App. C, Sec. II).
 *   n_spins >= 1; n_edges >= 0; edges: 2*n_edges int32 spin ids (u != v, no
 *   repeated pair); J: n_edges couplings; h: n_spins fields or NULL (must be
 *   NULL when q == 3); q: 2 (Ising) or 3 (Potts); flags: TN_DTYPE_*.
 *   On success *out owns a new context; free it with tn_destroy().
 *   Errors: TN_EINVAL on bad sizes/ids/q, TN_ENOMEM if host allocation fails.
 */
tn_status tn_build(tn_ctx **out, int32_t n_spins, int32_t n_edges,
                   const int32_t *edges, const float *J, const float *h,
                   int32_t q, uint32_t flags);

/*
 * Max-2-SAT (App. D): counting optimal assignments of an optimisation problem
 * on the same graph with the same kernels as the spin glass.  Literals are
 * signed 1-based variable ids: +(i+1) is x_i, -(i+1) is NOT x_i.  The cost of
 * an assignment is the number of violated clauses (l_u OR l_v).  Variable x_i
 * is spin i with x_i = true <-> sigma_i = +1 (state index 0).
 *
 * A clause's local tensor (-1 at its one violating pair of values, 0
 * elsewhere) equals, up to a constant, an Ising bond with coupling
 * -u_a u_b / 4 and fields -u_a / 4, -u_b / 4 (u = +1 when the literal is
 * false at sigma = +1, i.e. a negated literal, else -1).  Scaled by 4 these
 * are integers, so the network runs on the exact INT32 path and
 *   cost(x) = (E_ising(sigma) + n_clauses) / 4.
 *
 * tn_max2sat_couplings -- the Ising instance of a clause list (host only).
 *   n_vars >= 1, n_clauses >= 0; lits: 2*n_clauses literals, each variable id
 *   in 1..n_vars and the two variables of a clause distinct.  Clauses on the
 *   same pair of variables are merged into one edge (couplings summed).
 *   Writes *n_edges (<= n_clauses), edges (2*n_clauses capacity), J
 *   (n_clauses capacity) and h (n_vars).  Errors: TN_EINVAL.
 */
tn_status tn_max2sat_couplings(int32_t n_vars, int32_t n_clauses, const int32_t *lits,
                               int32_t *n_edges, int32_t *edges, float *J, float *h);

/*
 * tn_build_max2sat -- a context for a Max-2-SAT instance (arguments as
 *   above, flags: TN_DTYPE_AUTO or TN_DTYPE_I32).  It behaves like a tn_build
 *   context on the couplings of tn_max2sat_couplings, except that every
 *   energy it returns (tn_energy, tn_config, tn_count, tn_forward, the _batch
 *   forms and tn_batch_run) is the cost in violated clauses,
 *   (E_ising + n_clauses) / 4; sigma = +1 means true.  Batched calls take
 *   couplings from tn_max2sat_couplings of clause lists on the same variable
 *   pairs.  tn_gradient and tn_energy_noalloc return TN_ESTATE on it.
 *   Errors: TN_EINVAL as tn_max2sat_couplings.
 */
tn_status tn_build_max2sat(tn_ctx **out, int32_t n_vars, int32_t n_clauses,
                           const int32_t *lits, uint32_t flags);

/*
 * tn_order -- fix the pairwise contraction tree (Sec. III: the cost is
 *   exponential in the treewidth; regular lattices sweep row by row, general
 *   graphs use heuristics such as greedy).  Host only; plans the steps, the
 *   transposes and the device memory layout.
 *   TN_ORDER_SWEEP: seq holds seq_len distinct spin ids, eliminated in that
 *     order (spins left out follow in id order).
 *   TN_ORDER_GREEDY: seq ignored; `restarts` randomized greedy runs seeded by
 *     `seed`, the cheapest tree (time model over the steps) is kept.
 *   TN_ORDER_TREE: seq holds 2*(n_tensors-1) ids; leaves are tensors
 *     0..n_tensors-1 (see tn_leaf_count), step s creates tensor n_tensors+s.
 *   log2_peak / log2_ops (may be NULL) receive log2 of the largest tensor
 *   (elements) and of the total tropical multiply-adds of the plan.
 *   Errors: TN_EINVAL (bad sequence/tree), TN_ENOMEM (largest tensor above
 *   2^34 elements).
 */
tn_status tn_order(tn_ctx *ctx, int32_t method, const int32_t *seq, int32_t seq_len,
                   uint64_t seed, int32_t restarts, double *log2_peak, double *log2_ops);

/* Number of leaf tensors of the built network (one per edge, plus one per
 * isolated spin); the ids TN_ORDER_TREE refers to. */
int32_t tn_leaf_count(const tn_ctx *ctx);

/*
 * tn_set_couplings -- replace J (n_edges) and h (n_spins, or NULL = keep)
 *   without re-planning.  on_device = 0: host pointers (copied synchronously);
 *   1: device pointers on the context's device (copied on the context stream).
 *   INT32 contexts require integral values (TN_EINVAL otherwise, host only).
 */
tn_status tn_set_couplings(tn_ctx *ctx, const float *J, const float *h, int32_t on_device);

/* Make every launch of this context go to `cuda_stream` (a cudaStream_t,
 * NULL = legacy default stream).  The caller keeps the stream alive. */
tn_status tn_set_stream(tn_ctx *ctx, void *cuda_stream);

/*
 * tn_energy -- E_min by the tropical contraction (Sec. II).  Blocks until the
 *   result is on the host.  *E is exact for INT32 contexts; FP32 contexts
 *   accumulate in float (the returned double is the float result).
 */
tn_status tn_energy(tn_ctx *ctx, double *E);

/*
 * tn_config -- a ground state by argmax traceback (Sec. III): forward
 *   contraction keeping checkpoints, then a top-down walk of the tree that
 *   recomputes freed intermediates.  Ties take the first index in the order
 *   of the contracted legs (footnote in Sec. III).  sigma: n_spins int8
 *   (+1/-1 for Ising, 0..q-1 for Potts), host buffer; may be NULL when only
 *   the device-side result (tn_gradient) is wanted.  *E (may be NULL)
 *   receives E_min from the same forward pass.
 */
tn_status tn_config(tn_ctx *ctx, int8_t *sigma, double *E);

/*
 * tn_forward / tn_backward -- the two halves of tn_config, for autograd use.
 *   tn_forward runs the forward contraction keeping the traceback's
 *   checkpoints in the context's arena and returns E_min (*E may be NULL);
 *   tn_backward then runs the traceback (recomputing what was not kept) and
 *   leaves the state on the device for tn_gradient; sigma (n_spins int8,
 *   host, may be NULL) receives it as in tn_config.  tn_backward returns
 *   TN_ESTATE unless the last call on the context was tn_forward.
 */
tn_status tn_forward(tn_ctx *ctx, double *E);
tn_status tn_backward(tn_ctx *ctx, int8_t *sigma);

/*
 * tn_gradient -- derivatives of E_min at the last tn_config state (Sec. III):
 *   dE/dJ_e = -s_u s_v (Potts: -delta(s_u, s_v)), dE/dh_i = -s_i.  dJ has
 *   n_edges floats, dh n_spins floats (may be NULL).  on_device selects host
 *   or device buffers.  TN_ESTATE if tn_config has not run.
 */
tn_status tn_gradient(tn_ctx *ctx, float *dJ, float *dh, int32_t on_device);

/*
 * tn_count -- ground-state degeneracy with the counting tuples of Sec. II.
 *   n_primes in [1, 8] sets the range: the count is exact up to about
 *   2^(61*n_primes).  The residues are kept modulo ceil(61*n_primes/31)
 *   31-bit primes 2^31 - c in 4-byte planes when those fit in 9 planes
 *   (n_primes <= 4; TN_COUNT_61 forces the other form), else modulo n_primes
 *   61-bit primes 2^61 - c in 8-byte planes; one extra witness prime checks
 *   the reconstruction and TN_EOVERFLOW is returned when it disagrees.  When
 *   the planes do not fit in device memory the count runs once per 31-bit
 *   prime with a single plane (TN_COUNT_PASSES forces this).  limbs:
 *   little-endian 64-bit limbs of the count, capacity *n_limbs on input,
 *   limbs used on output.  ln_count (may be NULL): natural log of the count.
 *   *E (may be NULL): E_min of the same pass.
 */
tn_status tn_count(tn_ctx *ctx, int32_t n_primes, uint64_t *limbs, int32_t *n_limbs,
                   double *ln_count, double *E);

/*
 * tn_sample -- n_samples ground states drawn uniformly at random (Sec. III:
 *   fix the spins one at a time in `order`, each with its conditional
 *   probability of being in a ground state given the spins fixed before it).
 *   The conditional probabilities are exact ratios of degeneracy counts: a
 *   unit field on each fixed spin selects, among the ground states, those
 *   that agree with it, and tn_count_batch counts them (3 primes + witness),
 *   two candidates per sample and step, 16 samples per batch; n_spins steps.
 *   order: n_spins distinct spin ids, or NULL for 0..n_spins-1.  seed: sample
 *   s draws from a counter-based generator keyed by (seed, s, step), so the
 *   result does not depend on n_samples.  sigma: n_samples * n_spins values
 *   +-1, sample-major (host).  Requires tn_order, q == 2, an INT32 context
 *   (integral J and h: exact ties), couplings last set from the host.
 *   Errors: TN_EINVAL (arguments, q, dtype), TN_ESTATE (no order; counts that
 *   no ground state extends), TN_EOVERFLOW (a count beyond the primes),
 *   TN_ENOMEM / TN_ECUDA as tn_count_batch.
 */
tn_status tn_sample(tn_ctx *ctx, int32_t n_samples, uint64_t seed, const int32_t *order,
                    int8_t *sigma);

/*
 * Batches on one context: B coupling sets on the context's graph and order
 * (many disorder instances of one lattice).  Every kernel of the plan is
 * launched once for all B instances (instance = one grid dimension, each with
 * its own slice of the arena), the traceback runs one block per instance, and
 * the launch sequence is captured as a CUDA graph per (range, B).
 *   J: B*n_edges floats, instance-major; h: B*n_spins floats, required when
 *   the context was built with fields and NULL otherwise; on_device: 0 host
 *   pointers, 1 device pointers.  E: B doubles (host).  The arena grows to B
 *   times the single-instance plan (TN_ENOMEM if it does not fit).
 * tn_energy_batch -- E_min of each instance.
 * tn_config_batch -- E_min and the ground state (sigma: B*n_spins int8, host,
 *   may be NULL; same conventions as tn_config).
 * tn_count_batch -- E_min and degeneracy of each instance with the range of
 *   n_primes 61-bit primes + witness (residue planes as tn_count); limbs:
 *   B*limbs_per little-endian 64-bit limbs; status[b] (may be NULL) is TN_OK,
 *   TN_EOVERFLOW or TN_EINVAL (count needs more than limbs_per limbs).
 *   Returns the first non-OK status.
 */
tn_status tn_energy_batch(tn_ctx *ctx, int32_t B, const float *J, const float *h,
                          int32_t on_device, double *E);
tn_status tn_config_batch(tn_ctx *ctx, int32_t B, const float *J, const float *h,
                          int32_t on_device, double *E, int8_t *sigma);
tn_status tn_count_batch(tn_ctx *ctx, int32_t B, const float *J, const float *h,
                         int32_t on_device, int32_t n_primes, uint64_t *limbs, int32_t limbs_per,
                         double *E, int32_t *status);

/*
 * tn_batch_run -- many independent instances, each already built and ordered
 *   (possibly of different sizes).  Contexts with the same graph, dtype,
 *   energy map and contraction steps (compared exactly) are grouped and each
 *   group runs as one batch (as tn_count_batch with 3 primes + witness, or
 *   tn_energy_batch when limbs == NULL) on the group's first context.  All
 *   groups are queued before any is waited for, largest first, on a pool of
 *   non-blocking streams of the library (one stream while any group's context
 *   is profiling), after the work already queued on each first context's
 *   stream; the call returns when every result is on the host.  Outputs per
 *   instance k: E[k]; limbs[k*limbs_per ...]; and status[k].  Returns the
 *   first non-OK status, else TN_OK.
 */
tn_status tn_batch_run(int32_t B, tn_ctx *const *ctxs, double *E, uint64_t *limbs,
                       int32_t limbs_per, int32_t *status);

/*
 * Measurement hooks.  Every kernel launch of the context is counted; with
 * profiling enabled each launch is also bracketed by CUDA events on the
 * context stream.  tn_profile_get(kind): 0 leaves, 1 transpose, 2 gate
 * contraction, 3 max-plus GEMM, 4 traceback, 5 other, 6 fused gate chain,
 * -1 all; it synchronises
 * the stream and returns launches, total milliseconds (profiling only),
 * algorithmic bytes (operands read + result written, each once) and tropical
 * multiply-adds of those launches.  tn_profile_reset clears the counters.
 */
tn_status tn_set_profiling(tn_ctx *ctx, int32_t enable);
tn_status tn_profile_get(tn_ctx *ctx, int32_t kind, int64_t *launches, double *ms,
                         double *bytes, double *macs);
tn_status tn_profile_reset(tn_ctx *ctx);

/* Statistics of the current plan (any pointer may be NULL): number of
 * pairwise steps, transposes, device arena bytes for energy / config / count. */
tn_status tn_plan_info(const tn_ctx *ctx, int32_t *n_steps, int32_t *n_transposes,
                       int64_t *arena_energy, int64_t *arena_config, int64_t *arena_count);

/*
 * tn_plan_launches -- kernel launches of one execution of the lowered program
 *   (host only; Sec. III: which steps run as transposes + GEMMs and which as
 *   gate contractions or fused chains).  mode: 0 tn_energy, 1 tn_config
 *   (checkpoints kept, traceback included), 2 tn_count with 3 primes +
 *   witness.  counts: 7 int64 entries, indexed by the kinds of
 *   tn_profile_get (a counting GEMM or transpose is two launches: values and
 *   residue planes).  Errors: TN_EINVAL (arguments), TN_ESTATE (no order).
 */
tn_status tn_plan_launches(const tn_ctx *ctx, int32_t mode, int64_t *counts);

/*
 * tn_energy_noalloc -- E_min like tn_energy, for callers that cannot allocate
 *   device memory: code recording work inside a CUDA stream capture (where
 *   cudaMalloc is not allowed), frameworks whose caching allocator owns the
 *   whole device, and latency-critical loops that cannot pay for the device
 *   synchronisation that cudaMalloc / cudaFree imply.  The paper has no
 *   counterpart; it is an interface of this library only.
 *   ctx must be built and ordered (both are host-only and allocate no device
 *   memory).  J_dev (n_edges floats) and h_dev (n_spins floats; NULL only for
 *   instances built without fields) are device pointers the caller owns;
 *   E_dev receives E_min as one float in device memory; the work is queued
 *   on cuda_stream (NULL = legacy default stream) and the call does not wait
 *   for it.  INT32 contexts read J_dev / h_dev as integers (rounded).
 *   Scratch: a static 32 MiB device array inside libtn.so, held by every GPU
 *   that loads the library until the process exits.  A plan whose
 *   intermediates need more returns TN_ENOMEM with the size it needs
 *   (lattices up to about 20 x 20 fit).  The first call on a device looks up
 *   the array's device address (cudaGetSymbolAddress); make that first call
 *   before any stream capture.  No cudaMalloc, cudaFree, memory copy or
 *   allocating library routine is called: the leaf descriptors travel as
 *   kernel parameters, so the call only queues kernel launches on the
 *   stream.
 *   All calls share the one array and it keeps the last call's contents;
 *   every intermediate is written before it is read, so nothing needs
 *   clearing, but calls that overlap on the GPU (other streams, other host
 *   threads, other contexts) race on the scratch: serialise them.
 */
tn_status tn_energy_noalloc(tn_ctx *ctx, const float *J_dev, const float *h_dev, float *E_dev,
                            void *cuda_stream);

/*
 * tn_maxplus_gemm -- the batched max-plus GEMM of the pairwise steps (Eq. 2,
 *   Sec. III), exposed on raw device buffers for testing and measurement:
 *   C[b, m, n] = max_k (A[b, m, k] + B[b, k, n]).  dtype TN_DTYPE_F32 or
 *   TN_DTYPE_I32 (4-byte elements).  A is [batch][M][K] (transA = 0) or
 *   [batch][K][M] (transA = 1); B is [batch][K][N] (transB = 0) or
 *   [batch][N][K] (transB = 1); C is [batch][M][N]; all row-major, device
 *   memory owned by the caller.  Queued on cuda_stream, not waited for,
 *   except on the first call for a shape class (dtype, sizes, layout) made
 *   outside stream capture: that call times the candidate tile
 *   configurations on the stream (all give bit-identical C) and keeps the
 *   fastest for later calls and for the GEMM steps of contractions.  Set
 *   TN_NO_AUTOTUNE to skip the timing; TN_AUTOTUNE_CACHE names a file that
 *   keeps the choices across processes.
 *   Errors: TN_EINVAL (bad sizes, NULL), TN_ECUDA (launch); tn_last_error(NULL).
 */
tn_status tn_maxplus_gemm(int32_t dtype, int64_t batch, int64_t M, int64_t N, int64_t K,
                          const void *A, int32_t transA, const void *B, int32_t transB, void *C,
                          void *cuda_stream);

/* One-line reason for the last failing call on ctx (or of tn_build when ctx
 * is NULL).  Valid until the next call on the same context. */
const char *tn_last_error(const tn_ctx *ctx);

/* Free the context and its device memory.  NULL is ignored. */
void tn_destroy(tn_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */
