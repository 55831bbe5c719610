/*
 * apcg.h -- asynchronous device-scalar Jacobi-preconditioned CG for NVIDIA GB300.
 *
 * C ABI of libapcg.so.  Every call returns an apcg_status (0 = success,
 * negative = error), the convention of the paper's footnote to the core
 * stream-control listing (Sec. 3.1.1: every routine returns an error code).
 * On error, apcg_last_error_string() gives a per-thread message.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Pointers called "device" must point to memory the current CUDA device can
 *   read (cudaMalloc, cudaMallocAsync or PyTorch CUDA tensors); pointers called
 *   "host" must be ordinary host memory.  float64 vectors must be 16-byte
 *   aligned, float32 vectors 16-byte aligned as well (every CUDA and PyTorch
 *   allocation is).  Misaligned pointers return APCG_ERR_INVALID_ARG.
 * - The library never owns caller buffers.  apcg_vec / apcg_mat are
 *   non-owning views; the caller keeps the memory alive until the work that
 *   uses it has finished (apcg_ctx_synchronize, or a host accessor).
 * - Handles (contexts, scalars, vectors, matrices, plans) are owned by the
 *   caller and released with the matching *_destroy.  A destroy never
 *   blocks: device memory behind a handle is released only once every stream
 *   that used it is idle (Sec. 3.2.2, lifetime of managed objects).
 * - Arguments are validated before anything is enqueued.  Errors that arise
 *   on the device (a breakdown, a non-finite value, a bad diagonal) are
 *   recorded on the device and reported by the next call that synchronizes
 *   (a host accessor, apcg_ctx_synchronize, or a solver's result).
 * - A context argument of NULL selects the library's global-blocking
 *   context: the call waits for all prior work on every context and has
 *   completed when it returns (Sec. 3.1, global-blocking streams; Sec. 3.2.2,
 *   an Eval without a context).
 * - Thread safety: all entry points may be called from several host threads;
 *   operations on one context are ordered by the order of the calls.
 */
#ifndef APCG_H
#define APCG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define APCG_API __attribute__((visibility("default")))
#else
#define APCG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */

typedef int32_t apcg_status;

#define APCG_OK 0
#define APCG_ERR_INVALID_ARG (-1)  /* bad handle, size, pointer or alignment */
#define APCG_ERR_CUDA (-2)         /* a CUDA runtime call failed (message has the CUDA error) */
#define APCG_ERR_NO_MEMORY (-3)    /* device or host allocation failed */
#define APCG_ERR_BAD_DIAGONAL (-4) /* Jacobi: a diagonal entry is missing, zero or not finite */
#define APCG_ERR_TIMEOUT (-5)      /* a bounded device wait ran out */
#define APCG_ERR_UNSUPPORTED (-6)  /* valid request that this build does not support */
#define APCG_ERR_NOT_READY (-7)    /* query only: work still pending (never an error elsewhere) */
#define APCG_ERR_BREAKDOWN (-8)    /* a solver met (p, Ap) <= 0 or a non-finite value */

/* Message of the last failing call on this host thread (never NULL). */
APCG_API const char* apcg_last_error_string(void);
/* Library version as major*10000 + minor*100 + patch. */
APCG_API int32_t apcg_version(void);

/* ------------------------------------------------------------------ handles */

typedef struct apcg_ctx_s* apcg_ctx;
typedef struct apcg_scalar_s* apcg_scalar;
typedef struct apcg_vec_s* apcg_vec;
typedef struct apcg_mat_s* apcg_mat;
typedef struct apcg_cg_plan_s* apcg_cg_plan;
typedef uint64_t apcg_id;

typedef enum {
  APCG_STREAM_DEFAULT_BLOCKING = 0, /* asynchronous w.r.t. the host and every other context */
  APCG_STREAM_GLOBAL_BLOCKING = 1   /* waits for all prior work on every context, and
                                       completes before the launching call returns */
} apcg_stream_type;

typedef enum { APCG_ACCESS_READ = 1, APCG_ACCESS_WRITE = 2, APCG_ACCESS_READ_WRITE = 3 } apcg_access;

typedef enum {
  APCG_JOIN_DESTROY = 0, /* parent waits on every child, then the children are destroyed */
  APCG_JOIN_SYNC = 1,    /* parent waits on every child, then every child waits on the parent */
  APCG_JOIN_NO_SYNC = 2  /* parent waits on every child; children continue independently */
} apcg_join_mode;

typedef enum { APCG_F64 = 0, APCG_F32 = 1 } apcg_dtype;

/* ------------------------------------------------------------------ device contexts (Sec. 3.1) */

/*
 * Create a context on the current CUDA device owning a new non-blocking
 * stream (Sec. 3.1: a context is a device plus the stream it manages).
 * Stream type: APCG_STREAM_DEFAULT_BLOCKING.
 */
APCG_API apcg_status apcg_ctx_create(apcg_ctx* out);

/*
 * Create a context that borrows an existing CUDA stream (for example a
 * PyTorch stream), passed as its cudaStream_t value.  The stream is never
 * destroyed by the library and must outlive the context.
 */
APCG_API apcg_status apcg_ctx_create_from_stream(void* cuda_stream, apcg_ctx* out);

/* Select the stream type (Sec. 3.1).  Takes effect for the next call on the context. */
APCG_API apcg_status apcg_ctx_set_stream_type(apcg_ctx ctx, apcg_stream_type type);
APCG_API apcg_status apcg_ctx_get_stream_type(apcg_ctx ctx, apcg_stream_type* type);

/*
 * The cudaStream_t of the context, for launching caller kernels between
 * apcg_mark_intent_begin/end (marking listing example, Sec. 3.1.2).  The
 * caller must not destroy it or change its attributes.
 */
APCG_API apcg_status apcg_ctx_get_stream(apcg_ctx ctx, void** cuda_stream);

/*
 * Core stream control (listing "Core PetscDeviceContext Stream Control APIs",
 * Sec. 3.1.1): make `waiter` wait for all work enqueued on `waitee` so far;
 * ask whether all work of a context has finished (*idle = 1) without
 * blocking; block the host until all work of a context has finished.
 * apcg_ctx_synchronize also reports device-side errors recorded by work on
 * the context.
 */
APCG_API apcg_status apcg_ctx_wait_for_context(apcg_ctx waiter, apcg_ctx waitee);
APCG_API apcg_status apcg_ctx_query_idle(apcg_ctx ctx, int32_t* idle);
APCG_API apcg_status apcg_ctx_synchronize(apcg_ctx ctx);

/*
 * Fork and join (named among the paper's keywords; the paper does not spell
 * out their semantics, this is the library's reading): fork creates n child
 * contexts on the parent's device, with the parent's stream type, whose
 * streams start after everything enqueued on the parent so far.  Join makes
 * the parent wait for everything enqueued on each child, then applies `mode`.
 */
APCG_API apcg_status apcg_ctx_fork(apcg_ctx parent, int32_t n, apcg_ctx* children);
APCG_API apcg_status apcg_ctx_join(apcg_ctx parent, int32_t n, apcg_ctx* children, apcg_join_mode mode);

/* Destroy a context.  Pending work still completes; its stream is released afterwards. */
APCG_API apcg_status apcg_ctx_destroy(apcg_ctx ctx);

/* ------------------------------------------------------------------ memory IDs and intent marking (Sec. 3.1.2) */

/*
 * Register a memory region and obtain its object ID (listing "Memory
 * Registration API").  Registering a pointer that is already registered
 * returns the existing ID.  `ptr` may be a host or device address; `bytes`
 * is the size of the region.
 */
APCG_API apcg_status apcg_register_memory(const void* ptr, size_t bytes, apcg_id* id);
/* Look up the ID and size of a registered pointer (start address only). */
APCG_API apcg_status apcg_get_pointer_attributes(const void* ptr, apcg_id* id, size_t* bytes);
/* Forget a registration; pending marks on it still complete. */
APCG_API apcg_status apcg_unregister_memory(const void* ptr);

/*
 * Intent marking (listing "API For Marking Stream Dependencies"): bracket
 * every launch that accesses object `id` on context `ctx`.  Begin makes the
 * context's stream wait on exactly the earlier conflicting accesses made on
 * other contexts: the last write for a read; the last write and every read
 * since it for a write.  Same-context accesses keep program order and need
 * no wait; two reads are never ordered (the strong write-ordering rule,
 * Sec. 3.1.2).  End records the access.  `desc` is for debugging and may be
 * NULL.  Begin/end pairs for several IDs may be interleaved around one
 * launch.
 */
APCG_API apcg_status apcg_mark_intent_begin(apcg_ctx ctx, apcg_id id, apcg_access mode, const char* desc);
APCG_API apcg_status apcg_mark_intent_end(apcg_ctx ctx, apcg_id id, apcg_access mode, const char* desc);

/*
 * Host access to an object (the implicit synchronisation of accessors such
 * as VecGetArray, Sec. 3.3): block the host only until the accesses that
 * conflict with `mode` have finished -- the last write for a read, the last
 * write and all later reads for a write.
 */
APCG_API apcg_status apcg_host_access(apcg_id id, apcg_access mode);

/* ------------------------------------------------------------------ counters (profiling) */

typedef struct {
  int64_t kernel_launches;  /* kernels enqueued by the library (graph launches count their kernels) */
  int64_t graph_launches;   /* CUDA graph launches */
  int64_t waits_inserted;   /* cross-context event waits enqueued by marking */
  int64_t waits_elided;     /* conflicting accesses that needed no wait (already ordered or complete) */
  int64_t events_recorded;  /* events recorded at the end of marked launches */
  int64_t host_syncs;       /* host blocking points (accessors, synchronize, global-blocking calls) */
  int64_t d2h_copies;       /* device-to-host copies */
  int64_t d2h_bytes;
  int64_t h2d_copies;       /* host-to-device copies */
  int64_t h2d_bytes;
} apcg_counters;

APCG_API apcg_status apcg_get_counters(apcg_counters* out);
APCG_API apcg_status apcg_reset_counters(void);

/* ------------------------------------------------------------------ managed device scalars (Sec. 3.2) */

/*
 * A managed scalar is one float64 value that lives in device memory (a slot
 * of the library's scalar pool) and carries an object ID, so that producers
 * and consumers on different contexts are ordered by marking (Sec. 3.2: a
 * future for a value that stays on the device).  Only APCG_F64 is supported.
 * Creation enqueues nothing; the value is undefined until written.
 */
APCG_API apcg_status apcg_scalar_create(apcg_dtype dtype, apcg_scalar* out);
/* Enqueue value := v on ctx. */
APCG_API apcg_status apcg_scalar_set_async(apcg_ctx ctx, apcg_scalar s, double v);
/*
 * Host accessor (front() in the mixed-API CG example, Sec. 3.3): waits only
 * for the last write of the scalar, then copies it to *v.
 */
APCG_API apcg_status apcg_scalar_get(apcg_scalar s, double* v);
/* Device address of the slot (valid until apcg_scalar_destroy). */
APCG_API apcg_status apcg_scalar_device_ptr(apcg_scalar s, double** dptr);
/* The scalar's object ID, for apcg_mark_intent_* around caller kernels. */
APCG_API apcg_status apcg_scalar_id(apcg_scalar s, apcg_id* id);

/*
 * Scalar arithmetic evaluated on the device (what Eval(expr, dctx) launches,
 * Sec. 3.2.1-3.2.2): out := num / den, out := 1 / a, out := -a, out := a,
 * out := a * b, out := sqrt(a).  `out` may alias an input.
 */
APCG_API apcg_status apcg_scalar_div_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar num, apcg_scalar den);
APCG_API apcg_status apcg_scalar_recip_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a);
APCG_API apcg_status apcg_scalar_neg_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a);
APCG_API apcg_status apcg_scalar_copy_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a);
APCG_API apcg_status apcg_scalar_mul_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a, apcg_scalar b);
APCG_API apcg_status apcg_scalar_sqrt_async(apcg_ctx ctx, apcg_scalar out, apcg_scalar a);

/* Release the scalar; its slot is reused only after every access to it has finished. */
APCG_API apcg_status apcg_scalar_destroy(apcg_scalar s);

/* ------------------------------------------------------------------ vectors and matrices */

/*
 * Non-owning view of n contiguous elements at device pointer `dptr`
 * (Vec, Sec. 3.1.2).  The memory is registered (apcg_register_memory) and
 * the view takes that object ID.  n may be 0.
 */
APCG_API apcg_status apcg_vec_wrap(void* dptr, int64_t n, apcg_dtype dtype, apcg_vec* out);
APCG_API apcg_status apcg_vec_id(apcg_vec v, apcg_id* id);
APCG_API apcg_status apcg_vec_destroy(apcg_vec v);

/*
 * Non-owning view of a square or rectangular CSR matrix (AIJ, Sec. 4.1) in
 * device memory: rowptr[nrows+1] (int32, rowptr[0] = 0, non-decreasing),
 * col[nnz] (int32 in [0, ncols)), val[nnz] of `dtype`.  Column indices
 * need not be sorted, but the row sums are formed in storage order.
 * Wrapping checks nothing.  The CG, TFQMR and refinement plans check the
 * structure on the device when they are created (rowptr starts at 0, never
 * decreases and ends at nnz; column indices lie in [0, ncols)) and return
 * APCG_ERR_INVALID_ARG before any kernel reads through it.
 * The asynchronous operations (apcg_mat_mult_async, apcg_pc_jacobi_setup_async)
 * and the batched plans, which take raw CSR arrays, trust the structure:
 * call apcg_mat_validate first where it may be malformed.
 */
APCG_API apcg_status apcg_mat_csr_wrap(const int32_t* rowptr, const int32_t* col, const void* val, int32_t nrows,
                              int32_t ncols, int64_t nnz, apcg_dtype dtype, apcg_mat* out);
/* Check the structure on the host (copies the arrays back): rowptr monotone, columns in range. */
APCG_API apcg_status apcg_mat_validate(apcg_mat A);
APCG_API apcg_status apcg_mat_id(apcg_mat A, apcg_id* id);
APCG_API apcg_status apcg_mat_destroy(apcg_mat A);

/* ------------------------------------------------------------------ asynchronous vector / matrix operations (Sec. 3.3) */

/*
 * The *Async operations of Sec. 3.3 (VecDotAsync, VecNormAsync,
 * VecAXPYAsync, VecAYPX, VecScaleAsync, VecCopy, KSP_MatMultAsync,
 * KSP_PCApplyAsync).  Scalars are managed scalars read or written on the
 * device; each call marks its operands (read for inputs, write for outputs)
 * on `ctx` and enqueues one kernel.  Vectors must have equal lengths and
 * dtypes; only APCG_F64 vectors are supported by these generic operations.
 * Reductions are deterministic for a given length (fixed two-level order).
 */
APCG_API apcg_status apcg_vec_dot_async(apcg_ctx ctx, apcg_vec x, apcg_vec y, apcg_scalar out);    /* out := x'y */
APCG_API apcg_status apcg_vec_norm2_async(apcg_ctx ctx, apcg_vec x, apcg_scalar out);              /* out := ||x||_2 */
APCG_API apcg_status apcg_vec_axpy_async(apcg_ctx ctx, apcg_vec y, apcg_scalar a, int32_t negate,  /* y := y + (+-a) x */
                                apcg_vec x);
APCG_API apcg_status apcg_vec_aypx_async(apcg_ctx ctx, apcg_vec y, apcg_scalar b, apcg_vec x);     /* y := x + b y */
APCG_API apcg_status apcg_vec_scale_async(apcg_ctx ctx, apcg_vec y, apcg_scalar a);                /* y := a y */
APCG_API apcg_status apcg_vec_copy_async(apcg_ctx ctx, apcg_vec dst, apcg_vec src);                /* dst := src */
APCG_API apcg_status apcg_vec_set_async(apcg_ctx ctx, apcg_vec y, double v);                       /* y := v */
APCG_API apcg_status apcg_vec_pointwise_mult_async(apcg_ctx ctx, apcg_vec w, apcg_vec x,           /* w := x .* y */
                                          apcg_vec y);

/* y := A x (MatMult).  x has ncols elements, y has nrows; x and y must not alias. */
APCG_API apcg_status apcg_mat_mult_async(apcg_ctx ctx, apcg_mat A, apcg_vec x, apcg_vec y);
/* y := A x and out := x'y in one kernel (square A): the SpMV and the dot that follows it in CG. */
APCG_API apcg_status apcg_mat_mult_dot_async(apcg_ctx ctx, apcg_mat A, apcg_vec x, apcg_vec y, apcg_scalar out);

/*
 * Jacobi preconditioner (Sec. 4.1, diagonal scaling): setup writes
 * dinv := 1 ./ diag(A) (a missing diagonal entry counts as zero; a zero or
 * non-finite diagonal makes the next synchronizing call on ctx return
 * APCG_ERR_BAD_DIAGONAL); apply writes z := dinv .* r.
 */
APCG_API apcg_status apcg_pc_jacobi_setup_async(apcg_ctx ctx, apcg_mat A, apcg_vec dinv);
APCG_API apcg_status apcg_pc_jacobi_apply_async(apcg_ctx ctx, apcg_vec dinv, apcg_vec r, apcg_vec z);

/* ------------------------------------------------------------------ conjugate gradient solver (Sec. 3.3, Sec. 4.2) */

typedef enum {
  /* Scalars go to the host every iteration: (p,Ap) and (r,z),(r,r) are copied
     back and waited for, alpha and beta are computed on the host and passed
     by value -- the host-synchronous form the paper benchmarks against. */
  APCG_MODE_HOST_SYNC = 0,
  /* All scalars stay on the device; kernels are enqueued back to back and the
     host reads a 'done' flag once every check_every iterations. */
  APCG_MODE_ASYNC = 1,
  /* As ASYNC, with check_every iterations captured once as a CUDA graph and
     repeated by a device-side while loop (conditional graph node): one graph
     launch per solve and no host read until the solve ends. */
  APCG_MODE_ASYNC_GRAPH = 2,
  /* The whole solve in one kernel on one thread block (small systems). */
  APCG_MODE_PERSISTENT = 3,
  /* Library choice: PERSISTENT for small systems, ASYNC_GRAPH otherwise. */
  APCG_MODE_AUTO = 4
} apcg_mode;

typedef enum {
  APCG_CONVERGED = 0,
  APCG_NOT_CONVERGED = 1,
  APCG_BREAKDOWN = 2,
  APCG_BAD_DIAGONAL = 3 /* batched solves: this system has a zero, missing or non-finite diagonal entry */
} apcg_reason;

typedef struct {
  double rtol;          /* stop when ||r||_2 <= max(rtol * ||b||_2, atol) */
  double atol;
  int32_t max_it;       /* iteration cap; <= 0 selects 10 * n */
  int32_t check_every;  /* k: the test runs when the iteration count is a multiple of k (and at max_it); >= 1 */
  int32_t mode;         /* apcg_mode */
  int32_t history_len;  /* number of alpha/beta values to record (0 = none) */
  double* alpha_hist;   /* host [history_len] or NULL: alpha of iteration i at index i-1 */
  double* beta_hist;    /* host [history_len] or NULL: beta computed at the end of iteration i */
} apcg_cg_opts;

/* Fill opts with rtol 1e-8, atol 0, max_it 0, check_every 1, mode AUTO, no history. */
APCG_API apcg_status apcg_cg_opts_default(apcg_cg_opts* opts);

typedef struct {
  int32_t iters;            /* completed iterations */
  int32_t reason;           /* apcg_reason */
  double rr;                /* (r,r) of the recursively updated residual at the last convergence test */
  double bnorm;             /* ||b||_2 */
  double rel_res;           /* sqrt(rr) / bnorm (sqrt(rr) when b = 0), at the last convergence test */
  int64_t kernel_launches;  /* kernels this solve executed on the device */
} apcg_cg_result;

/*
 * Solve A x = b by Jacobi-PCG (textbook Hestenes-Stiefel CG with diagonal
 * scaling, Sec. 4.1-4.2; loop body in the order of the mixed-API CG example
 * of Sec. 3.3, with the standard initialisation r = b - A x0, z = D^-1 r,
 * p = z).  A is square float64 with a nonzero diagonal; x holds x0 on entry
 * and the iterate on exit.  Marks A and b read, x read-write.  One call is
 * apcg_cg_plan_create + apcg_cg_plan_solve + destroy: the set-up blocks the
 * host while it checks and converts the matrix, the solve once, at the end,
 * to fill *res.  Returns APCG_ERR_INVALID_ARG for a malformed CSR structure,
 * APCG_ERR_BAD_DIAGONAL for a zero, missing or non-finite diagonal entry, and
 * APCG_OK otherwise (a breakdown or the iteration cap is reported in
 * res->reason).
 */
APCG_API apcg_status apcg_cg_solve(apcg_ctx ctx, apcg_mat A, apcg_vec b, apcg_vec x, const apcg_cg_opts* opts,
                          apcg_cg_result* res);

/*
 * Reusable solver plan: set-up once per matrix and option set (structure
 * check, sliced-ELL copy, Jacobi diagonal, workspace, launch shapes, captured
 * graphs), then any number of solves.  Creation runs on the context's stream
 * and blocks the host until it is done; it returns APCG_ERR_INVALID_ARG for a
 * malformed CSR structure and APCG_ERR_BAD_DIAGONAL for a bad diagonal.  The
 * plan keeps non-owning references to A.  A plan's solves on one context are
 * ordered; the plan must not be used from two contexts at once.
 */
APCG_API apcg_status apcg_cg_plan_create(apcg_ctx ctx, apcg_mat A, const apcg_cg_opts* opts, apcg_cg_plan* out);
APCG_API apcg_status apcg_cg_plan_solve(apcg_cg_plan plan, apcg_vec b, apcg_vec x, apcg_cg_result* res);
/*
 * Enqueue a solve without waiting for it: the result stays on the device
 * until apcg_cg_plan_result() is called (which blocks until the solve ends).
 * History recording is not available through this pair.
 */
APCG_API apcg_status apcg_cg_plan_solve_async(apcg_cg_plan plan, apcg_vec b, apcg_vec x);
APCG_API apcg_status apcg_cg_plan_result(apcg_cg_plan plan, apcg_cg_result* res);
APCG_API apcg_status apcg_cg_plan_destroy(apcg_cg_plan plan);

/*
 * Kernel timing for performance reports: runs the set-up kernel once, then
 * `iters` iterations with each of the three iteration kernels launched on its
 * own between CUDA events recorded on the plan's context stream, and returns
 * their average durations in milliseconds (ms[0] = SpMV + (p,Ap), ms[1] =
 * updates + Jacobi + (r,z),(r,r), ms[2] = search-direction update).  The
 * iterations run regardless of convergence (iters must not exceed the
 * iteration count at which the system would break down: use a count well
 * below its convergence count).  x is overwritten with the iterate reached.
 */
APCG_API apcg_status apcg_cg_plan_profile(apcg_cg_plan plan, apcg_vec b, apcg_vec x, int32_t iters, float* ms);

/*
 * The sliced-ELL copy of the matrix that a plan's SpMV reads (slices of 32
 * consecutive rows stored column-major, each padded to its widest row; the
 * SpMV of Sec. 4.1's MatMult in a layout for 32-lane warps), for tests and
 * performance reports.  col_format says how each stored entry's column is
 * found:
 *   APCG_COLS_NONE      the plan holds no copy (whole-solve cluster mode, or a
 *                       stencil operator);
 *   APCG_COLS_INDEX     a 32-bit column index per stored entry;
 *   APCG_COLS_OFFSET16  a 16-bit offset from the row per stored entry (chosen
 *                       where every entry lies within 32767 of the diagonal);
 *   APCG_COLS_PATTERN   one list of column offsets per slice, shared by its 32
 *                       rows; a row that lacks one of them stores the value 0
 *                       there (chosen where every row's columns strictly
 *                       increase and these lists pad the slices by at most
 *                       1/16 more than their widest rows do: stencil
 *                       matrices).  The matrix values are then the only
 *                       per-entry stream.
 * Every format adds each row's entries in their CSR order.  group is the
 * SpMV's group size (entries per lane loaded before their FMAs; 0 = one at a
 * time), nslices the number of slices, padded the stored entries including
 * padding.  Plain host reads: never blocks.  Returns APCG_ERR_INVALID_ARG for
 * a NULL plan or out.
 */
#define APCG_COLS_NONE (-1)
#define APCG_COLS_INDEX 0
#define APCG_COLS_OFFSET16 1
#define APCG_COLS_PATTERN 2
typedef struct apcg_plan_layout {
  int32_t col_format; /* APCG_COLS_* */
  int32_t group;      /* SpMV group size, 0 = one entry at a time */
  int64_t nslices;    /* slices of 32 rows */
  int64_t padded;     /* stored entries including padding */
} apcg_plan_layout;
APCG_API apcg_status apcg_cg_plan_layout(apcg_cg_plan plan, apcg_plan_layout* out);

/*
 * The same solve for callers that hold the system in ordinary host memory:
 * copies rowptr/col/val/b/x to the device, solves on a library context, and
 * copies x back.  The copies are part of the call.
 */
APCG_API apcg_status apcg_cg_solve_host(int32_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col, const double* val,
                               const double* b, double* x, const apcg_cg_opts* opts, apcg_cg_result* res);

/*
 * Jacobi-PCG without any device allocation (the paper has no counterpart;
 * this entry point exists for callers that cannot allocate).  Some callers
 * cannot call cudaMalloc when they solve: a framework that reserved nearly
 * all device memory for its own pool leaves none for a library allocation,
 * and a real-time loop must not allocate after start-up because a device
 * allocation may synchronise the device and takes unbounded time.  This call
 * solves one system with the whole-solve cluster kernel (the PERSISTENT mode
 * of apcg_cg_solve) and keeps its scratch -- the Jacobi diagonal and the
 * solve's bookkeeping -- in a fixed array inside the library, which every GPU
 * that loads the library holds until the process exits.  It allocates no
 * device memory, creates no stream or context, and does no intent marking.
 *
 * cuda_stream: the caller's cudaStream_t (NULL selects the legacy default
 * stream); the work is ordered on it and the call blocks until it finishes.
 * rowptr/col/val, b, x: device CSR matrix and vectors as for apcg_cg_solve
 * (x holds x0 on entry).  opts: rtol, atol, max_it, check_every (mode and
 * history are ignored); NULL selects the defaults.  res: host, filled at exit.
 *
 * Limit: n <= 65536 rows (the size of the fixed array); larger n returns
 * APCG_ERR_INVALID_ARG before anything is enqueued.  Every call shares the
 * one array, which keeps the last call's contents (each call rewrites what it
 * reads): calls that overlap on the GPU -- on different streams or from
 * different host threads -- race and must not be issued.  Each call looks up
 * the array's address on the current device (cudaGetSymbolAddress, which
 * allocates nothing).  The call is synchronous: it ends by waiting for the
 * stream, so it must not be issued on a stream that is being captured.
 *
 * The CSR structure is checked on the device, reading rowptr[0..n] and
 * col[0..nnz) only, before any kernel reads through it: rowptr must start at
 * 0, never decrease and end at nnz, and every column must lie in [0, n);
 * otherwise the call returns APCG_ERR_INVALID_ARG.  A zero, missing or
 * non-finite diagonal entry returns APCG_ERR_BAD_DIAGONAL.  In both cases no
 * iteration runs and x keeps its entry value.
 */
APCG_API apcg_status apcg_cg_solve_noalloc(void* cuda_stream, int32_t n, int64_t nnz, const int32_t* rowptr,
                                           const int32_t* col, const double* val, const double* b, double* x,
                                           const apcg_cg_opts* opts, apcg_cg_result* res);

/* ------------------------------------------------------------------ mixed-precision iterative refinement */

/*
 * float64 iterative refinement around a float32 Jacobi-PCG (an extension of
 * the paper's float64 CG, Sec. 4.2; not in the paper).  float64 is kept only
 * for the outer residual r = b - A x, the update x += d and the convergence
 * norm; the inner PCG on A d = r runs in float32 (values, vectors, FMAs and
 * accumulation) from d = 0 until ||r_in|| <= rtol_inner ||(float) r||, or
 * max_inner iterations.  Outer stop: ||b - A x||_2 <= max(rtol ||b||_2, atol)
 * with the true residual in float64.
 *
 * A64: float64 CSR (device) used for the outer residual; may be NULL when the
 * float32 values are exact copies (the outer residual then widens them).
 * A32: float32 CSR with the same rowptr/col arrays; may be NULL, in which case
 * the plan keeps a round-to-nearest float32 copy of A64's values.
 */
typedef struct apcg_ir_plan_s* apcg_ir_plan;

typedef struct {
  double rtol;               /* outer relative tolerance (default 1e-10) */
  double atol;               /* outer absolute tolerance (default 0) */
  int32_t max_outer;         /* corrections (default 50) */
  int32_t max_inner;         /* inner iterations per correction (default 1000) */
  float rtol_inner;          /* inner relative tolerance (default 1e-4) */
  int32_t inner_check_every; /* inner convergence test every k iterations (default 1) */
  /* Single-system plans: the inner alpha and beta of the FIRST correction's
   * iterations 1..history_len (float32 values widened to double), written to
   * these host buffers by apcg_ir_plan_solve; iterations the correction does
   * not reach are NaN.  0 / NULL = none (default).  Batched plans ignore them. */
  int32_t history_len;
  int32_t pad;
  double* alpha_hist;
  double* beta_hist;
} apcg_ir_opts;

typedef struct {
  int32_t outer;            /* corrections applied */
  int32_t inner_total;      /* inner iterations summed over corrections */
  int32_t reason;           /* apcg_reason */
  int32_t inner_first;      /* inner iterations of the first correction (single-system plans) */
  double rel_res;           /* ||b - A x|| / ||b|| at exit (float64 true residual) */
  int64_t kernel_launches;  /* kernels executed */
} apcg_ir_result;

APCG_API apcg_status apcg_ir_opts_default(apcg_ir_opts* opts);
APCG_API apcg_status apcg_ir_plan_create(apcg_ctx ctx, apcg_mat A64, apcg_mat A32, const apcg_ir_opts* opts,
                                         apcg_ir_plan* out);
/* Solve A x = b (x holds x0 on entry).  Blocks once per correction to read two norms. */
APCG_API apcg_status apcg_ir_plan_solve(apcg_ir_plan plan, apcg_vec b, apcg_vec x, apcg_ir_result* res);
APCG_API apcg_status apcg_ir_plan_destroy(apcg_ir_plan plan);
/* The sliced-ELL copy the plan's SpMVs read (see apcg_cg_plan_layout; the float32 and float64 copies share it). */
APCG_API apcg_status apcg_ir_plan_layout(apcg_ir_plan plan, apcg_plan_layout* out);
/*
 * Kernel timing for performance reports, as apcg_cg_plan_profile: one outer
 * residual r = b - A x (float64, fused with the set-up of the inner solve),
 * then `iters` float32 inner iterations with each of the three iteration
 * kernels launched on its own between CUDA events, with no inner tolerance
 * (keep iters well below the inner convergence count).  ms[0] = the residual
 * kernel, ms[1..3] = the average durations of the inner SpMV + (p,Ap), the
 * updates + Jacobi + (r,z),(r,r) and the search-direction update, in
 * milliseconds.  x is read, not changed.  Blocks until the kernels are done.
 */
APCG_API apcg_status apcg_ir_plan_profile(apcg_ir_plan plan, apcg_vec b, apcg_vec x, int32_t iters, float* ms);
/*
 * Test hook for the bounded waits of the staged float32 SpMV (the inner SpMV
 * of a plan whose matrix takes per-slice offset lists with long rows: each
 * warp bulk-copies its next slice of values into shared memory and waits on
 * an mbarrier, about 0.16 s at most).  With on != 0 every copy announces 16 bytes
 * more than it moves, so every such wait runs out: the SpMV gives up, the
 * solve reports APCG_ERR_TIMEOUT (res->reason = APCG_BREAKDOWN) and the
 * context stays usable.  on = 0 restores normal operation.  Nothing faults:
 * the copies themselves are unchanged.  Returns APCG_ERR_UNSUPPORTED for a
 * plan without a staged SpMV.  Blocks until the plan's graph is re-captured.
 */
APCG_API apcg_status apcg_ir_plan_test_stall_copies(apcg_ir_plan plan, int32_t on);
/*
 * One application of the plan's float32 inner operator, for checking it
 * against a plain float32 product: w = A32 p by the very kernel the inner
 * iterations launch (the same sliced-ELL copy, column format, group size
 * and, where the plan stages values through shared memory, the staged form),
 * and gamma = (p, w) reduced in float32 as in the inner iteration's first
 * step (A2-A3 of the PCG loop of Sec. 3.3, in float32).
 *
 * p, w: float32 device vectors of the plan's length n (caller-owned, not
 * aliased).  gamma: host double, may be NULL.  Row i of w is the float32 sum
 * of its entries in CSR order, each added by a fused multiply-add.  The
 * plan's inner state is overwritten (every solve sets it up again).  Blocks
 * until w and gamma are ready.  Errors: APCG_ERR_INVALID_ARG for a NULL, wrongly
 * typed or wrongly sized vector; APCG_ERR_TIMEOUT if a bounded wait of the
 * staged SpMV ran out (w is then incomplete).
 */
APCG_API apcg_status apcg_ir_plan_inner_spmv(apcg_ir_plan plan, apcg_vec p, apcg_vec w, double* gamma);
APCG_API apcg_status apcg_ir_solve(apcg_ctx ctx, apcg_mat A64, apcg_mat A32, apcg_vec b, apcg_vec x,
                                   const apcg_ir_opts* opts, apcg_ir_result* res);

/* ------------------------------------------------------------------ scalar expressions (Eval) */

/*
 * Scalar expressions over managed scalars, evaluated on the device: the C-ABI
 * form of the expression templates and Eval() of Sec. 3.2.1 (templates
 * cannot cross a C interface).  An expression is a postfix list of terms:
 * APCG_EX_SCALAR pushes a managed scalar, APCG_EX_CONST a constant, a binary
 * operator pops b then a and pushes (a op b), a unary one pops a and pushes
 * op(a).  MIN/MAX follow fmin/fmax (a NaN operand yields the other one).
 *
 * apcg_expr_create "freezes" the expression (what Eval does): equal
 * subexpressions become one instruction (common-subexpression elimination),
 * subtrees of constants are folded where the host result equals the
 * device's (+ - * / sqrt neg recip abs min max; never sin cos exp log), and
 * only rewrites that keep every value are applied (x*1, 1*x, x/1, x-0, -(-x)).
 * Limits: at most 64 instructions after freezing and 16 distinct scalars;
 * the terms must leave exactly one value.  The expression references its
 * scalars (not copied); they must outlive its executions.
 */
typedef enum {
  APCG_EX_SCALAR = 0,
  APCG_EX_CONST = 1,
  APCG_EX_ADD = 2,
  APCG_EX_SUB = 3,
  APCG_EX_MUL = 4,
  APCG_EX_DIV = 5,
  APCG_EX_MIN = 6,
  APCG_EX_MAX = 7,
  APCG_EX_NEG = 8,
  APCG_EX_RECIP = 9,
  APCG_EX_SQRT = 10,
  APCG_EX_ABS = 11,
  APCG_EX_SIN = 12,
  APCG_EX_COS = 13,
  APCG_EX_EXP = 14,
  APCG_EX_LOG = 15
} apcg_expr_op;

typedef struct {
  int32_t op;     /* apcg_expr_op */
  int32_t pad;
  apcg_scalar s;  /* APCG_EX_SCALAR: the operand */
  double c;       /* APCG_EX_CONST: the value */
} apcg_expr_term;

typedef struct apcg_expr_s* apcg_expr;
APCG_API apcg_status apcg_expr_create(const apcg_expr_term* terms, int32_t nterms, apcg_expr* out);
APCG_API apcg_status apcg_expr_destroy(apcg_expr expr);
/* The frozen program: instruction and input counts, and (if text != NULL) one line per instruction. */
APCG_API apcg_status apcg_expr_describe(apcg_expr expr, int32_t* ninstr, int32_t* ninputs, char* text, size_t cap);
/* out := expr, one kernel launch (Execute of Sec. 3.2.1).  Marks the inputs read and out written. */
APCG_API apcg_status apcg_expr_execute_async(apcg_ctx ctx, apcg_expr expr, apcg_scalar out);
/* y += expr * x with the expression evaluated inside the AXPY kernel (no launch of its own). */
APCG_API apcg_status apcg_vec_axpy_expr_async(apcg_ctx ctx, apcg_vec y, apcg_expr expr, apcg_vec x);

/* ------------------------------------------------------------------ matrix-free stencil operators */

/*
 * A constant-coefficient stencil on an nx x ny x nz grid (x fastest, then y,
 * then z; row i = ix + nx (iy + ny iz)), applied without a matrix: the
 * finite-difference Laplace operators of Sec. 4.1, which the paper's JAX
 * comparison applies as a convolution (Sec. 4.4).  Row i of S x is
 *   sum over terms k of weights[k] * x[i + dx_k + nx (dy_k + ny dz_k)],
 * where a term whose neighbour (ix + dx_k, iy + dy_k, iz + dz_k) lies outside
 * the grid is dropped (Dirichlet boundary by elimination: S is the assembled
 * stencil matrix).  The terms are summed in ascending order of their linear
 * offset, the column order of an assembled row.
 *
 * offsets: host int32 [npts][3] = (dx, dy, dz), each within +-127, no offset
 * twice; weights: host float64 [npts], finite; 1 <= npts <= 27; nx ny nz
 * <= 2^31 - 1.  Both arrays are copied.  The object holds no device memory.
 */
typedef struct apcg_stencil_s* apcg_stencil;
APCG_API apcg_status apcg_stencil_create(int32_t nx, int32_t ny, int32_t nz, int32_t npts, const int32_t* offsets,
                                         const double* weights, apcg_stencil* out);
APCG_API apcg_status apcg_stencil_destroy(apcg_stencil stencil);
/* y = S x (device float64 [nx ny nz], not aliased).  Marks x read, y written. */
APCG_API apcg_status apcg_stencil_apply_async(apcg_ctx ctx, apcg_stencil stencil, apcg_vec x, apcg_vec y);
/*
 * A Jacobi-PCG plan on a stencil operator: the method, modes, options and
 * results of apcg_cg_plan_create, with the SpMV reading only x (no matrix
 * arrays).  The Jacobi diagonal is 1 / (the weight of the (0,0,0) term);
 * APCG_ERR_BAD_DIAGONAL if that term is missing, zero or not finite.  Modes:
 * HOST_SYNC, ASYNC, ASYNC_GRAPH (AUTO selects ASYNC_GRAPH; PERSISTENT returns
 * APCG_ERR_UNSUPPORTED: the whole-solve cluster kernel reads a CSR matrix).
 * Solve, profile and destroy with the apcg_cg_plan_* calls above.  The plan
 * copies the stencil; the stencil may be destroyed afterwards.
 */
APCG_API apcg_status apcg_cg_plan_create_stencil(apcg_ctx ctx, apcg_stencil stencil, const apcg_cg_opts* opts,
                                                 apcg_cg_plan* out);
/*
 * Mixed-precision refinement (the scheme of apcg_ir_plan_create) on a stencil
 * operator: the float64 outer residual uses the float64 weights, the float32
 * inner Jacobi-PCG the weights rounded to float32 and the Jacobi diagonal
 * 1 / (float) centre.  Without matrix arrays an inner iteration moves only
 * float32 vectors.  Solve and destroy with apcg_ir_plan_solve/destroy.
 * APCG_ERR_BAD_DIAGONAL if the centre term is missing, zero or not finite
 * (in float64 or float32).
 */
APCG_API apcg_status apcg_ir_plan_create_stencil(apcg_ctx ctx, apcg_stencil stencil, const apcg_ir_opts* opts,
                                                 apcg_ir_plan* out);

/* ------------------------------------------------------------------ TFQMR */

/*
 * Transpose-free quasi-minimal residual (Freund 1993), the paper's second
 * solver (Sec. 4.3: two matrix-vector products and about twice the inner
 * products of a CG iteration; for nonsymmetric and indefinite systems too),
 * with the Jacobi preconditioner applied on the left: the method runs on
 * M = D^-1 A and D^-1 b, D = diag(A), with the shadow residual r* = r0.
 *
 * A: square float64 CSR with a nonzero diagonal (need not be symmetric).
 * b, x: device float64 [n], 16-byte aligned; x holds x0 on entry and the
 * iterate on exit.  Marks A and b read, x read-write.
 *
 * opts (apcg_cg_opts): rtol, atol, max_it (<= 0: 10 n), check_every k, mode,
 * history.  Modes: HOST_SYNC, ASYNC, ASYNC_GRAPH as for CG; PERSISTENT runs
 * the whole solve in one thread-block-cluster launch and takes n <= 16384
 * (APCG_ERR_UNSUPPORTED above that, or where the device cannot schedule the
 * cluster); AUTO selects PERSISTENT where it applies, else ASYNC_GRAPH.  The
 * persistent form reads the CSR arrays in place for the whole solve.
 * Convergence test, every k iterations and at max_it: Freund's bound
 * sqrt(2i + 1) tau_i <= max(rtol ||D^-1 b||, atol), tau_i the quasi-residual
 * norm after iteration i (two half-steps); a quasi-residual of exactly zero
 * stops at once.  alpha_hist[i-1] receives alpha of iteration i, beta_hist[i-1]
 * the beta formed at its end.
 *
 * Result (apcg_cg_result): iters, reason, rr = (sqrt(2 iters + 1) tau)^2 (the
 * bound, squared), bnorm = ||D^-1 b||, rel_res = bound / bnorm.  Returns
 * APCG_ERR_BAD_DIAGONAL for a zero, missing or non-finite diagonal entry
 * (at plan creation); a breakdown ((v, r*) = 0, (r*, w) = 0 or a non-finite
 * scalar) or the iteration cap is reported in res->reason.
 */
typedef struct apcg_tfqmr_plan_s* apcg_tfqmr_plan;
APCG_API apcg_status apcg_tfqmr_plan_create(apcg_ctx ctx, apcg_mat A, const apcg_cg_opts* opts,
                                            apcg_tfqmr_plan* out);
/* Solve with a plan; blocks until the solve ends. */
APCG_API apcg_status apcg_tfqmr_plan_solve(apcg_tfqmr_plan plan, apcg_vec b, apcg_vec x, apcg_cg_result* res);
APCG_API apcg_status apcg_tfqmr_plan_destroy(apcg_tfqmr_plan plan);
/* The sliced-ELL copy the plan's SpMV reads (see apcg_cg_plan_layout). */
APCG_API apcg_status apcg_tfqmr_plan_layout(apcg_tfqmr_plan plan, apcg_plan_layout* out);
/* One-shot form of create + solve + destroy. */
APCG_API apcg_status apcg_tfqmr_solve(apcg_ctx ctx, apcg_mat A, apcg_vec b, apcg_vec x, const apcg_cg_opts* opts,
                                      apcg_cg_result* res);

/* ------------------------------------------------------------------ batched solves (many independent systems) */

/*
 * Many independent SPD systems solved together by Jacobi-PCG (the paper's
 * method applied to each system; batching itself is not in the paper).  The
 * systems are concatenated row-wise: system s owns rows sys_row_off[s] ..
 * sys_row_off[s+1]-1; rowptr (device, int32 [N+1], N = sys_row_off[nsys])
 * holds nnz positions over the whole concatenation; col (device, int32) holds
 * column indices local to each system (0 .. n_s-1); val (device, float64).
 * b and x are concatenated the same way (device, float64 [N]; x holds x0 on
 * entry).  Each system must have at most 65536 rows.
 *
 * Every system is solved by one thread-block cluster that runs the whole
 * solve in one launch with a per-system convergence test; clusters take
 * systems longest first from a device work queue.  Systems are grouped into
 * size classes (powers of two in n), and each class has a launch shape
 * (CTAs per cluster, threads per CTA, rows per thread) picked by the built-in
 * table or by apcg_batch_plan_tune.  All class launches of a solve form one
 * CUDA graph whose branches run concurrently.
 *
 * opts: rtol, atol, max_it (per system; <= 0 selects 10 n_s), check_every;
 * mode, alpha_hist and beta_hist are ignored.  history_len > 0 makes every
 * solve record alpha and beta of iterations 1..history_len of EVERY system on
 * the device (2 * nsys * history_len doubles of plan memory), read with
 * apcg_batch_plan_history.  sys_row_off is host memory; it is copied.
 */
typedef struct apcg_batch_plan_s* apcg_batch_plan;

typedef struct {
  int32_t iters;   /* completed iterations of this system (refinement: inner iterations summed) */
  int32_t reason;  /* apcg_reason */
  double rel_res;  /* ||r|| / ||b|| at the last convergence test (CG: recursive residual;
                      refinement: the float64 true residual b - A x) */
  int32_t outer;   /* refinement: corrections applied; 0 for CG */
  int32_t pad;
} apcg_batch_result;

APCG_API apcg_status apcg_batch_plan_create(apcg_ctx ctx, int32_t nsys, const int32_t* sys_row_off,
                                            const int32_t* rowptr, const int32_t* col, const double* val,
                                            const apcg_cg_opts* opts, apcg_batch_plan* out);
/*
 * Batched mixed-precision refinement: every system is solved by the scheme of
 * apcg_ir_plan_create (float64 true residual and update, float32 Jacobi-PCG
 * for each correction started from zero, Sec. 3.3's CG in the inner loop), all
 * of it inside the system's cluster in one launch.  val (float64) serves the
 * outer residual and val32 (float32) the inner solves; either may be NULL:
 * a NULL val widens val32 (exact when the float32 values are the matrix), a
 * NULL val32 rounds val to nearest in the kernel.  The inner Jacobi diagonal
 * is the float32 one.  opts NULL selects apcg_ir_opts_default.  The plan is
 * solved, tuned and destroyed with the apcg_batch_plan_* calls below.
 */
APCG_API apcg_status apcg_batch_ir_plan_create(apcg_ctx ctx, int32_t nsys, const int32_t* sys_row_off,
                                               const int32_t* rowptr, const int32_t* col, const double* val,
                                               const float* val32, const apcg_ir_opts* opts,
                                               apcg_batch_plan* out);
/* Solve all systems; results (host [nsys]) may be NULL.  Blocks until done when results != NULL. */
APCG_API apcg_status apcg_batch_plan_solve(apcg_batch_plan plan, const double* b, double* x,
                                           apcg_batch_result* results);
/*
 * Autotuner: for every size class, time each candidate launch shape on the
 * class's own systems (b given, x0 = 0, a private x) and keep the fastest.
 * Writes up to `cap` lines "n_lo n_hi C threads rows_per_thread ms" into
 * `table` (may be NULL).  Blocks until done.
 */
APCG_API apcg_status apcg_batch_plan_tune(apcg_batch_plan plan, const double* b, char* table, size_t cap);
/*
 * The alpha and beta (Sec. 3.3's CG scalars) of iterations 1..history_len of
 * system `sys` in the last solve of a float64 batched plan created with
 * opts.history_len > 0; iterations the system did not reach are NaN.  alpha,
 * beta: host buffers of history_len doubles (either may be NULL).  Waits for
 * the plan's last solve.  APCG_ERR_INVALID_ARG for a plan without history
 * (refinement plans have none) or sys outside [0, nsys).
 */
APCG_API apcg_status apcg_batch_plan_history(apcg_batch_plan plan, int32_t sys, double* alpha, double* beta);
APCG_API apcg_status apcg_batch_plan_destroy(apcg_batch_plan plan);

/* One-shot form of create + solve + destroy. */
APCG_API apcg_status apcg_cg_solve_batched(apcg_ctx ctx, int32_t nsys, const int32_t* sys_row_off,
                                           const int32_t* rowptr, const int32_t* col, const double* val,
                                           const double* b, double* x, const apcg_cg_opts* opts,
                                           apcg_batch_result* results);

/* ------------------------------------------------------------------ measurement support */

/*
 * Launch floors on ctx's stream (the paper has no counterpart; the benchmark
 * reports them beside the per-iteration times of latency-bound solves), each
 * averaged over `reps` repetitions, in microseconds of host wall time:
 * us[0] one empty kernel launched and waited for; us[1] a graph of three
 * dependent empty kernels launched and waited for; us[2] an 8-byte
 * device-to-host copy and wait; us[3] the three-kernel graph launched back to
 * back (per graph, one wait at the end).  us: host [4].  Blocks.
 */
APCG_API apcg_status apcg_launch_floor(apcg_ctx ctx, int32_t reps, double* us);
/*
 * Measured float64 FMA throughput of this GPU (the paper has no counterpart;
 * the benchmark divides the float64 rate of its SpMV by it): a kernel of
 * independent fma chains on every SM, at full occupancy, timed with CUDA
 * events on ctx's stream; *gflops = 2 x FMAs / the fastest of `reps`
 * launches (after one warm-up launch), in GFLOP/s.  Allocates an output
 * buffer from the library pool.  Blocks.
 */
APCG_API apcg_status apcg_fp64_fma_peak(apcg_ctx ctx, int32_t reps, double* gflops);

/* ------------------------------------------------------------------ host-only simulation of the marking rules */

/*
 * A simulator of intent marking that never touches a GPU, driving the same
 * dependency tracker as the real contexts.  It exists so that the ordering
 * rules of Sec. 3.1.2 can be tested on machines without a GPU.  Contexts are
 * numbered 0..nctx-1; each apcg_sim_op is one launch that accesses `nids`
 * objects with the given modes; each simulated launch gets sequence number
 * 1, 2, ... on its context.  apcg_sim_complete marks every launch of `ctx`
 * with sequence <= seq as finished.  The log lists the waits the tracker
 * inserted as "w<-c@s" (context w waits for launch s of context c), one per
 * line, and the elided ones as "w..c@s".
 */
typedef struct apcg_sim_s* apcg_sim;
APCG_API apcg_status apcg_sim_create(int32_t nctx, apcg_sim* out);
APCG_API apcg_status apcg_sim_op(apcg_sim sim, int32_t ctx, int32_t nids, const apcg_id* ids, const int32_t* modes);
APCG_API apcg_status apcg_sim_complete(apcg_sim sim, int32_t ctx, uint64_t seq);
APCG_API apcg_status apcg_sim_log(apcg_sim sim, char* buf, size_t len);
APCG_API apcg_status apcg_sim_destroy(apcg_sim sim);

#ifdef __cplusplus
}
#endif

#endif /* APCG_H */
