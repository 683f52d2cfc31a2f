/* pc.h - C ABI of libpc: polyhedral-complex extraction from ReLU networks by
 * edge subdivision (Berzins, "Polyhedral Complex Extraction from ReLU Networks
 * using Edge Subdivision", ICML 2023), on one GB300 (sm_103a).
 *
 * What is computed (Sections 3.3, 3.4 and 4): a ReLU MLP with layers
 *   x^(l) = ReLU(W^(l) x^(l-1) + b^(l)),  l = 1..L   (Eq. 4)
 * and a box domain [lo, hi]^D induce a polyhedral complex whose cells are named
 * by sign vectors (Eq. 1-2).  The library returns the complex's vertices,
 * edges and the sign vector of every vertex.  Every neuron of every layer
 * (the output layer included) contributes one folded hyperplane; each is
 * processed in turn by steps (1)-(5) of Section 4.2.
 *
 * Conventions
 *   - W^(l) is (out x in), row-major, z = W x + b.
 *   - Network parameters are passed as ONE flat float64 array, in the order
 *     W1, b1, W2, b2, ..., WL, bL (each W row-major).
 *   - Sign-vector entries: the m = 2D box facets first (entry 2d: x_d - lo_d,
 *     entry 2d+1: hi_d - x_d; + means inside), then the neurons layer by
 *     layer.  Entry j is stored as a 2-bit code at bits 2*(j % 32) of 64-bit
 *     word j / 32: 00 = 0 (on the hyperplane), 01 = +, 10 = -.
 *   - Device arrays are structure-of-arrays with a leading dimension ld
 *     (the current capacity): coordinates X[d * ld + v], sign words
 *     SIG[w * ld + v], edge endpoints U[e] and V[e] = U[ld + e].
 *
 * Ownership and errors
 *   - A context owns every device buffer it returns; pointers stay valid until
 *     the next pc_extract or pc_destroy on that context.
 *   - Inputs are copied at the start of pc_extract; the caller may free them
 *     when the call returns.
 *   - Every call returns a pc_status; nothing aborts the process.  On an
 *     error pc_last_error() gives a message and the context is left empty
 *     but usable.
 *   - A context is not thread-safe: one call at a time per context.
 */
#ifndef PC_H_
#define PC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pc_ctx pc_ctx;

typedef enum {
  PC_OK = 0,
  PC_ERR_INVALID = 1,     /* bad argument or unsupported shape */
  PC_ERR_OOM = 2,         /* device allocation failed or budget exceeded */
  PC_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  PC_ERR_DEGENERATE = 4,  /* genericity violated (strict mode only) */
  PC_ERR_PAIRING = 5,     /* a splitting 2-face did not occur exactly twice */
  PC_ERR_TOO_LARGE = 6,   /* memory estimate above the budget (server) */
  PC_ERR_TIMEOUT = 7,     /* a bounded device-side wait ran out */
  PC_ERR_NO_TAPE = 8,     /* pc_backward without keep_tape */
  PC_PENDING = 9          /* server: request not finished yet */
} pc_status;

typedef enum {
  PC_PREC_FP32 = 0,   /* FP32 values, FP32 sign decisions */
  PC_PREC_MIXED = 1,  /* FP32/3xTF32 bulk, FP64 re-evaluation of every sign
                         whose FP32 value is within its error bound */
  PC_PREC_FP64 = 2    /* FP64 values throughout */
} pc_precision;

typedef enum {
  PC_EXEC_PERSISTENT = 0, /* one cooperative kernel per layer, grid barriers */
  PC_EXEC_STEPWISE = 1    /* one kernel per step and neuron */
} pc_exec;

typedef enum {
  PC_GEMM_TENSOR = 0,        /* tcgen05 tensor-core product for layers with
                                widths <= 128 (FP32 and mixed precision), SIMT
                                FP32 otherwise; the first layer (K = D) is
                                always FP64 FMA.  Operands split in three TF32
                                pieces (exact for FP32), six MMAs: FP32
                                accuracy */
  PC_GEMM_SIMT = 1,          /* SIMT FP32 FMA for every layer */
  PC_GEMM_TENSOR_3XTF32 = 2  /* tensor cores, two-piece 3xTF32 (three MMAs,
                                about 22 bits per product; the value error
                                scale is widened to match) */
} pc_gemm;

typedef enum {
  PC_PAIR_DEFERRED = 0, /* 2-faces keyed by a 64-bit fingerprint of their full
                           sign vector, paired at the second occurrence in
                           one 128-bit atomic; every pairing is then checked
                           exactly from the two new vertices' sign vectors,
                           and a failed check (a fingerprint collision)
                           repeats the extraction with PC_PAIR_INLINE */
  PC_PAIR_INLINE = 1    /* 32-bit tag; the second occurrence compares the
                           full sign vectors before it pairs */
} pc_pairing;

typedef struct {
  int precision;          /* pc_precision */
  int exec;               /* pc_exec */
  int keep_tape;          /* record the interpolation tape for pc_backward */
  int strict;             /* return PC_ERR_DEGENERATE on any genericity violation */
  int64_t init_vcap;      /* initial vertex capacity (grown x2 on overflow) */
  int64_t init_ecap;      /* initial edge capacity */
  int64_t mem_budget_bytes; /* 0 = no limit */
  double filter_kappa;    /* PC_PREC_MIXED: re-evaluate a sign in FP64 when
                             |z| <= kappa * (rms FP32 error estimate of z) */
  int polish;             /* Newton polish (values in float-float arithmetic,
                             about 44 bits) of every vertex whose rms
                             coordinate error estimate exceeds polish_tol *
                             box diameter: 1 on, 0 off, -1 on in
                             PC_PREC_MIXED only */
  double polish_tol;      /* relative to the box diameter (default 1e-6) */
  int timers;             /* record CUDA events around each layer's kernels */
  int gemm;               /* pc_gemm: layer-start product of FP32 values */
  int pairing;            /* pc_pairing: how step 5 matches the two
                             occurrences of a splitting 2-face */
  int canonical;          /* 1: return the result in canonical order:
                             vertices sorted by their packed sign words (word
                             0 most significant, unsigned), edges renumbered
                             and sorted by (smaller, larger) endpoint, so that
                             two extractions give identical arrays; the
                             values and error estimates follow the vertices.
                             Not with keep_tape (PC_ERR_INVALID at pc_create):
                             the tape refers to creation order */
  int prune;              /* 1: pruning during edge subdivision (Section
                             5.4.2) for level-set extraction: after each layer
                             but the last, edges whose vertices have the same
                             signs w.r.t. all future neurons (FP64 forward
                             pass at the vertex) are dropped, and at the end
                             the vertices without an edge; the result keeps
                             the output neuron's zero set and its
                             neighbourhood.  Not with keep_tape */
  int debug_barrier_timeout; /* testing only (0 in normal use): 1 makes every
                             grid barrier of the persistent kernel wait for one
                             arrival more than the grid has, with a spin limit
                             of 4096 polls, so that the wait runs out and the
                             extraction returns PC_ERR_TIMEOUT; exercises the
                             bounded-wait error path without hanging the GPU.
                             No effect in PC_EXEC_STEPWISE (no grid barrier) */
  double filter_kappa_audit; /* PC_PREC_MIXED, 0 = off: values with
                             filter_kappa < |z| / estimate <= this are also
                             evaluated in FP64 at the exact vertex, but only
                             recorded (pc_diagnostics: signs the filter would
                             have missed, and their largest margin), never
                             written back, so the extraction is the one that
                             filter_kappa alone gives */
} pc_options;

/* Fills *opt with defaults (mixed precision, persistent execution,
 * filter_kappa 12, polish in mixed precision with polish_tol 1e-6, tensor-core
 * layer products). */
void pc_default_options(pc_options *opt);

/* Creates a context on CUDA device `device`.  opt may be NULL (defaults). */
pc_status pc_create(pc_ctx **out, int device, const pc_options *opt);
pc_status pc_destroy(pc_ctx *ctx);

/* Optional device allocator used for every buffer of the context (for
 * example a framework's caching allocator).  alloc returns a device pointer
 * or NULL; stream is the cudaStream_t of the call.  Without it the context
 * uses cudaMallocAsync / cudaFreeAsync. */
typedef void *(*pc_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*pc_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
pc_status pc_set_allocator(pc_ctx *ctx, pc_alloc_fn alloc, pc_free_fn free_fn, void *user);

/* Edge subdivision (Section 4.2): extracts the complex of the network on the
 * box.  widths: host array of L+1 ints (widths[0] = D).  params: flat float64
 * parameters (layout above), host or device memory.  box_lo/box_hi: host
 * arrays of D doubles.  stream: cudaStream_t (NULL = legacy default stream).
 * Blocks until the result is ready (one device->host status read).
 * Limits: 1 <= D <= 8 (D <= 10 in libpc_d10.so, the same sources built with
 * PC_MAX_D=10), widths <= 256, 2D + sum(widths[1..L]) <= 1024.
 * Returns PC_ERR_PAIRING / PC_ERR_DEGENERATE (strict) when genericity fails. */
pc_status pc_extract(pc_ctx *ctx, int L, const int32_t *widths, const double *params,
                     const double *box_lo, const double *box_hi, void *stream);

/* Edge subdivision on a polyhedral domain instead of a box (Section 4.1: a
 * bounded domain given by m affine half-spaces; Section 5.2 suggests a
 * simplex, whose vertex and edge counts grow linearly and quadratically with
 * D instead of exponentially).  The domain is {x : c - A x >= 0}: A (m x D,
 * row-major) and c (m) are host float64 arrays.  Its 1-skeleton is the
 * caller's: X0 (nv0 x D, row-major, float64) and E0 (ne0 x 2 int32 vertex
 * indices), host arrays, copied at the start of the call.  Sign-vector
 * entry i < m is facet i (c_i - A_i x, + inside); the neurons follow at
 * m, m + 1, ...  Facet i of an initial vertex is 0 when
 * |c_i - A_i x| <= 1e-12 (|c_i| + sum_d |A_id x_d|), + otherwise.  As for
 * the box, a facet's zero is perturbed only toward + in step (5).
 * The domain must be a simple polytope and the skeleton complete:
 *   - every vertex inside and on exactly D facets;
 *   - every edge joins two distinct vertices sharing D - 1 facets;
 *   - no edge twice, D edges at every vertex;
 *   - a full-dimensional bounding box;
 *   - D + 1 <= m and m + neurons <= 1024.
 * Otherwise the call returns PC_ERR_INVALID before any device work.  The
 * coordinate tolerance of the polish is relative to the diameter of the
 * skeleton's bounding box.  Every other option, output and error is as for
 * pc_extract. */
pc_status pc_extract_domain(pc_ctx *ctx, int L, const int32_t *widths, const double *params, int m,
                            const double *A, const double *c, int64_t nv0, const double *X0, int64_t ne0,
                            const int32_t *E0, void *stream);

/* The checks pc_extract_domain makes on a domain and its skeleton (host
 * only, no device or context needed): PC_OK or PC_ERR_INVALID. */
pc_status pc_check_domain(int D, int m, const double *A, const double *c, int64_t nv0, const double *X0,
                          int64_t ne0, const int32_t *E0);

/* Counts of the last extraction: vertices, edges, 64-bit words per sign
 * vector, input dimension D, and sign-vector entries (2D + neurons). */
pc_status pc_counts(pc_ctx *ctx, int64_t *n_vertices, int64_t *n_edges, int32_t *sig_words,
                    int32_t *dim, int32_t *n_entries);

/* Vertex coordinates, float64, SoA X[d * ld + v].  *dev and *ld receive the
 * device array (either may be NULL); if out != NULL the D x nV block is copied
 * to out (host or device memory, row d at out + d * nV). */
pc_status pc_vertices(pc_ctx *ctx, const double **dev, int64_t *ld, double *out);

/* Edges, int32 vertex indices U[e], V[e] = U[ld + e]; out (nullable) receives
 * 2 x nE (row 0 = first endpoints, row 1 = second endpoints). */
pc_status pc_edges(pc_ctx *ctx, const int32_t **dev, int64_t *ld, int32_t *out);

/* Packed sign vectors, SIG[w * ld + v]; out (nullable) receives S x nV. */
pc_status pc_signvectors(pc_ctx *ctx, const uint64_t **dev, int64_t *ld, uint64_t *out);

/* The last layer's pre-activations at every vertex of the last extraction
 * (the network output before ReLU): widths[L] x nV values, row j at
 * out + j * nV, float32 (PC_PREC_FP32 / PC_PREC_MIXED) or float64
 * (PC_PREC_FP64); host or device memory.  Vertices on an output neuron's
 * zero set hold exactly 0 for it. */
pc_status pc_values(pc_ctx *ctx, void *out);

/* FP32 and mixed precision: per-vertex error estimates of the last
 * extraction, nV floats each (host or device memory, either may be NULL).
 * value_scale[v] = rho: the rms FP32 error of the vertex's last-layer value
 * z_j is about ||W_j||_2 rho + 2^-25 |b_j|.  coord_rms[v]: rms estimate of the
 * coordinate error accumulated by FP32 crossing parameters (before the
 * polish). */
pc_status pc_error_estimates(pc_ctx *ctx, float *value_scale, float *coord_rms);

/* Per-neuron counters of the last extraction, host array of n_neurons x 8
 * int64: vertices before, edges before, splitting edges, 2-face keys, paired
 * faces, FP64 re-evaluations, undecidable signs, genericity violations. */
pc_status pc_stats(pc_ctx *ctx, int64_t *out, int n_neurons);

/* Adjoint of the vertex coordinates with respect to the parameters, through
 * the interpolation formula of step (4) and the per-layer forward products of
 * step (1).  grad_x: D x nV float64 (row d at grad_x + d * nV), host or device.
 * grad_params: flat float64 array in the parameter layout, host or device;
 * overwritten.  Needs keep_tape = 1 at extraction (else PC_ERR_NO_TAPE). */
pc_status pc_backward(pc_ctx *ctx, const double *grad_x, double *grad_params, void *stream);

/* k-cell counts of the last extraction's complex (Section 4.1: the k-faces
 * by perturbing the zeros of the (k-1)-faces, a box facet's zero only toward
 * the inside): f_out[k] for k = 0..D (f_out needs n >= D + 1 entries;
 * f_out[D] is the number of regions), and optionally the Euler
 * characteristic sum (-1)^k f_k (1 for the subdivided box).  Runs on the
 * device; deduplicates the cells of each level by 64-bit fingerprints with
 * an exact check of every duplicate (PC_ERR_PAIRING on a collision,
 * PC_ERR_DEGENERATE on a non-generic cell).  Blocks until done. */
pc_status pc_cell_counts(pc_ctx *ctx, int64_t *f_out, int n, int64_t *euler);

/* The face poset of the last extraction's complex (Section 4.1: a k-cell
 * has D - k zeros in its sign vector; perturbing one zero to + or - (a box
 * facet's zero only to +, the inside) gives a (k+1)-cell that contains it,
 * its parent).  Builds on the device, and keeps in the context until the
 * next extraction: level 0 = the vertices (in pc_vertices order), level 1 =
 * the edges (in pc_edges order), level k >= 2 = the k-cells by perturbation,
 * deduplicated by 64-bit fingerprints with every duplicate compared word by
 * word; and for every cell of level k < D its parents, the cells of level
 * k + 1 obtained by perturbing its zeros in entry order, + before -.
 * PC_ERR_PAIRING on a fingerprint collision or a vertex perturbation that is
 * no edge, PC_ERR_DEGENERATE on a non-generic cell, PC_ERR_OOM.  Blocks. */
pc_status pc_build_poset(pc_ctx *ctx);

/* Level k of the poset (0 <= k <= D): *n_cells cells and *n_parents
 * parent incidences (0 for k = D).  Non-null outputs are filled (host or
 * device memory): cells, n_cells x S packed sign words, cell-major (cell i
 * at cells + i * S, the code layout of pc_signvectors); for k < D the
 * parents as CSR, row_ptr (n_cells + 1) and parents (n_parents indices into
 * level k + 1).  PC_ERR_INVALID before pc_build_poset or after the next
 * extraction. */
pc_status pc_poset_level(pc_ctx *ctx, int k, int64_t *n_cells, int64_t *n_parents, uint64_t *cells,
                         int64_t *row_ptr, int64_t *parents);

/* Diagnostics of the last extraction, up to n int64 values: kernel launches
 * (cumulative over the context's life), capacity growths, polished vertices,
 * exact-zero pre-activations, FP64-undecidable signs, vertex / edge / hash
 * capacities, device bytes held, CTAs of the persistent kernel, extractions
 * repeated with inline pairing after a failed fingerprint check (cumulative),
 * FP64 re-decisions that changed the FP32 sign (PC_PREC_MIXED), and the
 * largest |z| / (FP32 error estimate of z) among those, times 1000 and
 * rounded up (the filter re-decides every |z| <= filter_kappa x estimate, so
 * a margin near filter_kappa means a flip close to the filter's edge); then,
 * with filter_kappa_audit, the FP32 signs beyond filter_kappa that FP64 shows
 * wrong (each one an error the filter let through) and their largest
 * margin, times 1000. */
pc_status pc_diagnostics(pc_ctx *ctx, int64_t *out, int n);

/* With opt.timers: device time in ms of the last extraction's kernels,
 * out_ms[2l] = layer-start forward product of layer l, out_ms[2l+1] = the
 * neuron loop of layer l, out_ms[2L] = coordinate polish (-1 where not
 * measured). */
pc_status pc_kernel_times(pc_ctx *ctx, double *out_ms, int n);

/* ---------------------------------------------------------------------------
 * Serving: a persistent request loop around pc_extract (no counterpart in the
 * paper).  Requests arrive at any time (pc_server_submit copies the inputs
 * and returns at once).  A request whose memory estimate exceeds
 * request_max_bytes is rejected with PC_ERR_TOO_LARGE; the others queue in
 * FIFO order.  max_slots worker threads each own one context and one CUDA
 * stream; a free worker admits the head of the queue once the running
 * requests' estimates plus its own fit mem_budget_bytes, so requests that
 * arrive while others run are admitted as slots and memory free up and their
 * kernels overlap on the device; each context grows its arrays on overflow.
 * max_slots = 1 is the plain per-request path (FIFO, one at a time, same
 * kernels).  Times are seconds on the server's clock (since creation).
 * Thread-safe: submit / poll / wait_all may be called from any thread. */
typedef struct pc_server pc_server;

typedef struct {
  int max_slots;               /* concurrent requests (1 = plain FIFO path) */
  int precision;               /* pc_precision of every request */
  int exec;                    /* pc_exec of every request */
  int polish;                  /* pc_options.polish of every request */
  int keep_outputs;            /* keep each result's arrays in host memory */
  int64_t mem_budget_bytes;    /* admission limit on the summed estimates */
  int64_t request_max_bytes;   /* larger estimates are rejected */
} pc_server_options;

typedef struct {
  pc_status status;            /* PC_PENDING until finished */
  int64_t n_vertices, n_edges;
  double arrival_s, start_s, finish_s;
  int64_t est_bytes;           /* admission estimate (pc_estimate_bytes) */
  int slot;                    /* worker that ran it (-1 if rejected) */
  int64_t held_bytes;          /* device bytes its worker's context held after it */
} pc_result;

/* Device-memory estimate of one extraction: vertices ~ 1.2 N^D / D! for
 * generic ReLU nets with N neurons (the measured range is 0.4 - 1.2), edges ~
 * D x vertices, doubled for capacity growth.  -1 on bad input. */
int64_t pc_estimate_bytes(int L, const int32_t *widths);
/* Defaults: 8 slots, mixed precision, stepwise execution, no polish, 160 GiB
 * budget, 64 GiB per request.  A slot whose context holds more than 8 GiB
 * after a request frees its buffers (the next request allocates again). */
void pc_server_default_options(pc_server_options *opt);
pc_status pc_server_create(pc_server **out, int device, const pc_server_options *opt);
/* Inputs are host arrays (copied): widths L+1, params flat float64, box D. */
pc_status pc_server_submit(pc_server *s, int L, const int32_t *widths, const double *params,
                           const double *box_lo, const double *box_hi, uint64_t *id);
/* PC_OK with the final result, PC_PENDING while queued or running. */
pc_status pc_server_poll(pc_server *s, uint64_t id, pc_result *out);
/* Blocks until no request is queued or running (PC_ERR_TIMEOUT after
 * timeout_s seconds). */
pc_status pc_server_wait_all(pc_server *s, double timeout_s);
/* keep_outputs: copies a finished request's arrays to host memory: X (D x nV,
 * row d at X + d * nV), E (2 x nE), SIG (S x nV); any may be NULL. */
pc_status pc_server_outputs(pc_server *s, uint64_t id, double *X, int32_t *E, uint64_t *SIG);
/* Error message of a failed request ("" if none); valid until release. */
const char *pc_server_error(pc_server *s, uint64_t id);
/* Forgets a finished request (frees its kept outputs). */
pc_status pc_server_release(pc_server *s, uint64_t id);
/* Peak and current summed estimates of admitted requests. */
pc_status pc_server_stats(pc_server *s, int64_t *peak_bytes, int64_t *in_use_bytes);
/* Stops the workers (queued requests are dropped) and frees everything. */
pc_status pc_server_destroy(pc_server *s);

/* Allocation-free extraction, for callers that cannot allocate device
 * memory while they run (inside a custom memory pool or an allocator
 * callback, on real-time paths that forbid cudaMalloc because it can
 * synchronise the device, or under a fixed device-memory reservation).  The
 * paper has no counterpart: it is the same edge subdivision as pc_extract,
 * without a context, run one kernel per step.
 *
 * Inputs: widths (host, L+1), params (flat float64, host or device), box_lo /
 * box_hi (host, D), precision (pc_precision; mixed precision polishes as
 * pc_extract does by default).  Outputs, caller-owned device arrays with the
 * caller's capacities as leading dimensions: X (D x cap_v float64, X[d*cap_v +
 * v]), E (2 x cap_e int32, second endpoints at E + cap_e), SIG (S x cap_v
 * uint64, S = (2D + neurons + 31) / 32); *n_vertices / *n_edges (host).
 * Blocks until done.
 *
 * Alignment: cap_e must be a multiple of 4 and E must start on a 16-byte
 * boundary (the edge pass reads both endpoint rows with 16-byte loads); X
 * and SIG must be 8-byte aligned.  Otherwise the call returns PC_ERR_INVALID
 * before any device work.
 *
 * All other working memory is one static device array of about 10.6 MB
 * inside the library, held on every GPU that loads it until the process
 * exits.  Limits: cap_v <= 16384, cap_e <= 65536, layer widths <= 32, at most
 * 512 neurons and 16384 parameters; beyond them the call returns
 * PC_ERR_TOO_LARGE, and an extraction that outgrows the capacities returns
 * PC_ERR_OOM (nothing grows; the next call starts afresh).  Step (5) pairs
 * every 2-face with a full sign-vector comparison before it pairs (the
 * inline form of pc_pairing), so no check after the extraction is needed.  The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.  The first call on a device looks
 * up the scratch array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  Every
 * call shares the one scratch array and it keeps the last call's contents
 * (each call resets what must start empty); calls that overlap on the GPU
 * (on different streams or host threads) race with each other.
 * Other returns: PC_ERR_INVALID (bad argument), PC_ERR_PAIRING (genericity
 * failure), PC_ERR_TIMEOUT, PC_ERR_CUDA. */
pc_status pc_extract_noalloc(int L, const int32_t *widths, const double *params, const double *box_lo,
                             const double *box_hi, int precision, double *X, int32_t *E, uint64_t *SIG,
                             int64_t cap_v, int64_t cap_e, int64_t *n_vertices, int64_t *n_edges,
                             void *stream);

/* Message of the last error on this context ("" if none). */
const char *pc_last_error(pc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* PC_H_ */
