/*
 * tci_b300.h -- C ABI of the B300 (sm_103a) tensor-contraction library.
 *
 * The tensor handle, the label-based contraction and the manipulation calls
 * follow the Tensor Computing Interface (TCI) of arXiv 2512.23917, App. C
 * ("Type system", "Core functions", "Environment variables").  The
 * effective-Hamiltonian, Lanczos, block-sparse and batched-TEBD entry points
 * are extensions built on that contraction; each says where its definition
 * comes from.
 *
 * Conventions for every entry point
 *  - Return value: a tci_status.  TCI_OK on success; otherwise nothing was
 *    launched for a validation error, and tci_last_error(ctx) holds a one-line
 *    message.  No C++ exception crosses this boundary.
 *  - Asynchrony: device work is enqueued on the context's stream and the call
 *    returns without waiting, except calls that hand a host scalar back
 *    (tci_norm, tci_normalize, tci_close, tci_lanczos), which synchronise the
 *    stream before returning.
 *  - Memory: "device pointer" means memory of the context's device; "host
 *    pointer" means ordinary host memory (pinned memory is faster but not
 *    required).  Tensors created by tci_allocate / tci_zeros / tci_copy and
 *    contraction outputs the library creates are OWNED (freed by
 *    tci_tensor_free / tci_clear); tci_tensor_wrap creates a BORROWED view
 *    that the library never frees.  Owned memory is stream-ordered: it comes
 *    from a per-device pool on the context's stream and is released in order
 *    on the stream it was allocated on (which must still exist when the
 *    tensor is freed).  Work another stream does on an owned tensor must be
 *    complete, or waited for by that stream, before the tensor is freed.
 *  - Layout: shapes and strides are in elements, row-major when strides are
 *    omitted (last bond fastest), int64.
 *  - Thread safety: a context must not be used from two host threads at once.
 */
#ifndef TCI_B300_H
#define TCI_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum {
  TCI_OK = 0,
  TCI_ERR_INVALID_ARG = 1,     /* NULL pointer, negative size, bad enum          */
  TCI_ERR_SHAPE = 2,           /* shapes/orders/strides incompatible             */
  TCI_ERR_LABEL = 3,           /* repeated label in one operand, count mismatch  */
  TCI_ERR_DTYPE = 4,           /* element types differ or are not supported      */
  TCI_ERR_UNSUPPORTED = 5,     /* valid request outside what is implemented      */
  TCI_ERR_ALLOC = 6,           /* device allocation failed                       */
  TCI_ERR_CUDA = 7,            /* a CUDA runtime/driver call failed              */
  TCI_ERR_TIMEOUT = 8,         /* a bounded device wait expired (kernel status)  */
  TCI_ERR_INVALID_CONTEXT = 9  /* NULL or destroyed context                      */
} tci_status;

/* Element types: TCI elem_t (App. C.1, Tab. II) restricted to real/complex
 * IEEE types.  Complex values are interleaved (re, im). */
typedef enum { TCI_F32 = 0, TCI_F64 = 1, TCI_C64 = 2, TCI_C128 = 3 } tci_dtype;

/* Arithmetic used for real contractions (context-wide; see
 * tci_context_set_precision).
 *  TCI_PREC_NATIVE     : the element type's own arithmetic (FP64 FMA for F64).
 *  TCI_PREC_SPLIT_BF16 : each operand is split into three bfloat16 pieces
 *                        (hi, mid, lo; hi+mid+lo == fl32(x)); the six piece
 *                        products with i+j <= 2 run on the tcgen05 tensor
 *                        cores with FP32 accumulation in tensor memory, and
 *                        K-chunks of the accumulation are promoted to FP64.
 *  TCI_PREC_SPLIT_BF16_3 : same pieces, only the three products with
 *                        i+j <= 1 (about 2x faster, ~5e-6 relative error). */
typedef enum {
  TCI_PREC_NATIVE = 0,
  TCI_PREC_SPLIT_BF16 = 1,
  TCI_PREC_SPLIT_BF16_3 = 2
} tci_precision;

typedef struct tci_context_s* tci_context;   /* TCI context_handle_t */
typedef struct tci_tensor_s* tci_tensor;     /* TCI TenT              */
typedef struct tci_heff_plan_s* tci_heff_plan;
typedef struct tci_bs_plan_s* tci_bs_plan;
typedef struct tci_tebd_plan_s* tci_tebd_plan;

/* TCI "version" (App. C.2, Miscellaneous): specification version "M.m".
 * Returns a static string; never fails. */
const char* tci_version(void);

/* Human-readable name of a status code (static string). */
const char* tci_status_string(tci_status s);

/* Message of the last failed call on ctx (or of the last failed call with a
 * NULL/invalid context when ctx is NULL).  Static/thread-local storage; valid
 * until the next call on the same context. */
const char* tci_last_error(tci_context ctx);

/* ---------------------------------------------------------------- context */
/* TCI "create_context" (App. C.2, Miscellaneous): bind a context to CUDA
 * device `device` and stream `stream` (a cudaStream_t; NULL = the legacy
 * default stream).  Reads TCI_VERBOSE (App. C.3) once: 0 silent, 1 one line
 * per call on stderr, 2 adds the call's device time (this synchronises).
 * Also reads TCI_FAULT_ALLOC (extension, for tests of the out-of-memory
 * path): "n:k" makes the context's pooled device allocation number n
 * (0-based, counted from creation) fail k times in a row on the host, as if
 * the device were out of memory, before the pool is asked; k = 1 exercises
 * the trim-and-retry path (the call succeeds), k >= 2 makes the call return
 * TCI_ERR_ALLOC.  The device is never touched by the injection.
 * On failure *ctx is set to NULL.  Errors: INVALID_ARG, CUDA. */
tci_status tci_create_context(tci_context* ctx, int device, void* stream);

/* TCI "destroy_context": release the context and everything it owns;
 * *ctx becomes NULL.  Tensors created on it must be freed first. */
tci_status tci_destroy_context(tci_context* ctx);

/* Change the stream later calls enqueue on (extension of create_context's
 * implementation-defined parameters). */
tci_status tci_context_set_stream(tci_context ctx, void* stream);

/* Select the arithmetic of real contractions (see tci_precision).  Plans
 * (tci_heff_plan_create, tci_bs_plan_create) capture the mode at creation. */
tci_status tci_context_set_precision(tci_context ctx, tci_precision p);
tci_status tci_context_get_precision(tci_context ctx, tci_precision* p);

/* Accumulation granularity of the split-BF16 tensor-core GEMM (a tuning
 * knob of the plan): hi*hi products are accumulated in FP32 tensor memory
 * for chunk_k of contraction depth, the cross products for xchunk_k, before
 * being folded into an error-free FP32 double-float sum.  Smaller chunks are
 * more accurate and cost more epilogue work.  Defaults 256 / 1024 (measured
 * relative error of the chi = 2048 H_eff matvec: 4.3e-7; 128 / 1024: 2.2e-7).
 * Errors: INVALID_ARG unless 32 | chunk_k and chunk_k | xchunk_k. */
tci_status tci_context_set_split_chunks(tci_context ctx, int chunk_k, int xchunk_k);

/* Limit of each bounded device wait of the tensor-core kernels (extension;
 * the paper has no counterpart), in nanoseconds; 0 restores the default of
 * 2 s.  A wait that expires makes the kernel record a status word, let its
 * in-flight copies and MMAs land, free its tensor memory and return; the
 * next synchronising call reports TCI_ERR_TIMEOUT (once) and the context
 * stays usable.  Tiny limits exist to exercise that path in tests.  Plans
 * that replay a captured CUDA graph (block-sparse, TEBD) keep the limit in
 * force when their graph was captured.
 * Errors: INVALID_CONTEXT. */
tci_status tci_context_set_wait_limit(tci_context ctx, uint64_t limit_ns);

/* Measured FP64 FMA rate of the context's device (extension; the paper has
 * no counterpart): one kernel of 4 blocks of 256 threads per SM, each thread
 * running 8 independent FP64 FMA chains for `iters` iterations, timed with
 * CUDA events on the context's stream; *gflops (host) receives the best of
 * three launches after a warm-up, as 2 flops per FMA.  It is the FP64
 * roofline denominator of the benchmark.  Synchronises; allocates and frees
 * a small device buffer.  Errors: INVALID_ARG (NULL gflops, iters < 1),
 * ALLOC, CUDA, INVALID_CONTEXT. */
tci_status tci_probe_fp64_rate(tci_context ctx, int iters, double* gflops);

/* Block the host until all work queued on the context's stream finished;
 * maps a sticky device error or a kernel timeout status to CUDA/TIMEOUT. */
tci_status tci_synchronize(tci_context ctx);

/* ---------------------------------------------------------------- tensors */
/* Borrowed view of existing device memory `data` (TCI TenT, App. C.1):
 * dtype, order (0..8), shape[order], strides[order] in elements (NULL =
 * row-major contiguous).  The library never frees `data`.
 * Errors: INVALID_ARG (order > 8, negative dims/strides, NULL data with
 * nonzero size), DTYPE. */
tci_status tci_tensor_wrap(tci_context ctx, tci_dtype dtype, int order, const int64_t* shape,
                           const int64_t* strides, void* data, tci_tensor* out);

/* TCI "allocate" / "zeros" (App. C.2, Construction): owned, row-major,
 * uninitialised / zero-filled.  Errors: INVALID_ARG, DTYPE, ALLOC. */
tci_status tci_allocate(tci_context ctx, tci_dtype dtype, int order, const int64_t* shape,
                        tci_tensor* out);
tci_status tci_zeros(tci_context ctx, tci_dtype dtype, int order, const int64_t* shape,
                     tci_tensor* out);

/* TCI "eye" (App. C.2, Tensor construction): *out = a new owned n x n
 * identity tensor (ones on the main diagonal, zeros elsewhere) of dtype.
 * Errors: INVALID_ARG (n < 0, NULL out), DTYPE, ALLOC, CUDA. */
tci_status tci_eye(tci_context ctx, tci_dtype dtype, int64_t n, tci_tensor* out);

/* TCI "fill" (App. C.2, Tensor construction): *out = a new owned row-major
 * tensor of the given shape with every element equal to re + i im (im is
 * ignored for real dtypes).  Errors: as tci_allocate. */
tci_status tci_fill(tci_context ctx, tci_dtype dtype, int order, const int64_t* shape, double re, double im,
                    tci_tensor* out);

/* TCI "cplx_conj" (App. C.2, Tensor manipulation): elementwise complex
 * conjugation.  In place: t is conjugated (a real tensor is left unchanged;
 * a lazy layout is materialised first).  _to: *out = a new owned conjugated
 * copy (a deep copy for real dtypes).  Errors: INVALID_ARG, ALLOC, CUDA. */
tci_status tci_cplx_conj(tci_context ctx, tci_tensor t);
tci_status tci_cplx_conj_to(tci_context ctx, tci_tensor in, tci_tensor* out);

/* TCI "to_cplx" (App. C.2, Tensor manipulation): *out = a new owned complex
 * tensor of in's shape (F32 -> C64, F64 -> C128, zero imaginary parts); a
 * complex input gives a deep copy.  Errors: INVALID_ARG, ALLOC, CUDA. */
tci_status tci_to_cplx(tci_context ctx, tci_tensor in, tci_tensor* out);

/* TCI "diag" (App. C.2, Tensor linear algebra): a first-order input of
 * length n becomes the n x n matrix with it on the main diagonal; a
 * second-order input [d0, d1] gives its main diagonal, of length
 * min(d0, d1).  In place: t's shape and storage are replaced.  _to: *out is
 * a new owned tensor.  Errors: SHAPE (order other than 1 or 2), INVALID_ARG,
 * ALLOC, CUDA. */
tci_status tci_diag(tci_context ctx, tci_tensor t);
tci_status tci_diag_to(tci_context ctx, tci_tensor in, tci_tensor* out);

/* TCI "copy" (deep copy): *out becomes a new owned, row-major tensor with
 * the same logical elements as `in` (strided inputs are materialised). */
tci_status tci_copy(tci_context ctx, tci_tensor in, tci_tensor* out);

/* TCI "move": transfer metadata and storage of *from into a new handle
 * *to; *from is left an empty order-0 tensor with no storage. */
tci_status tci_move(tci_context ctx, tci_tensor from, tci_tensor* to);

/* TCI "clear": release the storage (if owned) and reset t to an empty
 * order-0 tensor with no storage. */
tci_status tci_clear(tci_context ctx, tci_tensor t);

/* Release the handle (and owned storage); *t becomes NULL.  Enqueued work
 * that uses the storage must have been synchronised by the caller. */
tci_status tci_tensor_free(tci_tensor* t);

/* Host transfer, the analogue of TCI "to_range" / "assign_from_range"
 * (App. C.2, Construction) for a contiguous host range in the tensor's
 * logical row-major element order.  `host` holds size(t) elements of t's
 * dtype.  tci_to_host synchronises; tci_from_host is stream-ordered but
 * blocks until `host` may be reused. */
tci_status tci_to_host(tci_context ctx, tci_tensor t, void* host);
tci_status tci_from_host(tci_context ctx, tci_tensor t, const void* host);

/* TCI read-only queries (App. C.2): order, shape, size (element count),
 * size_bytes; plus strides, dtype and the device address of element 0. */
tci_status tci_order(tci_context ctx, tci_tensor t, int* order);
tci_status tci_shape(tci_context ctx, tci_tensor t, int64_t* shape);      /* order entries */
tci_status tci_strides(tci_context ctx, tci_tensor t, int64_t* strides);  /* order entries */
tci_status tci_size(tci_context ctx, tci_tensor t, int64_t* size);
tci_status tci_size_bytes(tci_context ctx, tci_tensor t, int64_t* bytes);
tci_status tci_get_dtype(tci_context ctx, tci_tensor t, tci_dtype* dtype);
tci_status tci_data(tci_context ctx, tci_tensor t, void** data);

/* TCI "reshape" (App. C.2, Tensor manipulation; Sec. II.B.1):
 * metadata-only change to `order`/`new_shape` (same element count).  The
 * element order is the logical row-major order of the current shape; when
 * the current strides cannot express the new shape (e.g. after a lazy
 * transpose) the tensor is first materialised row-major on the device
 * (owned storage).  Errors: SHAPE (element count differs). */
tci_status tci_reshape(tci_context ctx, tci_tensor t, int order, const int64_t* new_shape);
/* Out-of-place: *out is a new handle; it shares storage with `in` when no
 * materialisation is needed (borrowed view) and owns a copy otherwise. */
tci_status tci_reshape_to(tci_context ctx, tci_tensor in, int order, const int64_t* new_shape,
                          tci_tensor* out);

/* TCI "transpose" (Eq. 1, Sec. II.B.1; App. C.2): B_{i_pi(0)..} = A_{i_0..}
 * with new_order[k] = the old bond that becomes bond k.  In place it is
 * lazy: only shape/stride metadata is permuted; contraction reads the
 * permuted operand in place.  Errors: INVALID_ARG (not a permutation). */
tci_status tci_transpose(tci_context ctx, tci_tensor t, const int* new_order);
/* Out-of-place: *out is a new owned row-major tensor holding the permuted
 * elements (a device permute-copy). */
tci_status tci_transpose_to(tci_context ctx, tci_tensor in, const int* new_order, tci_tensor* out);

/* TCI "contract" (App. C.2, Tensor linear algebra; Eq. C_IJ = sum_S A_IS
 * B_SJ of Sec. II.B.2).  Labels: one char per bond (string API) or int32
 * lists (tci_contract_l, lengths = the operands' orders and nc).  A label in
 * both a and b and not in c is summed; c's labels give its bonds and their
 * order; an empty c label list makes an order-0 (scalar) c.
 *  *c == NULL      : a new owned row-major c is created.
 *  *c is a tensor  : it must have c's shape and dtype (else SHAPE/DTYPE,
 *                    unless owned, in which case it is re-allocated); it may
 *                    alias a and/or b (the result is computed into scratch
 *                    first, then placed).
 * Both operands must have the same dtype.  Real F64/F32 contractions use the
 * context precision; complex ones use native arithmetic.
 * A label in a, b and c at once is a batch bond: every slice of it is
 * contracted on its own (C_IJB = sum_S A_ISB B_SJB), all slices in one
 * launch (real operands under a split precision: one grouped tensor-core
 * launch; otherwise native arithmetic).
 * Errors: LABEL (repeated label in one operand, count mismatch, dimension
 * mismatch), UNSUPPORTED (a free label missing from c), DTYPE, ALLOC, CUDA. */
tci_status tci_contract(tci_context ctx, tci_tensor a, const char* labels_a, tci_tensor b,
                        const char* labels_b, tci_tensor* c, const char* labels_c);
tci_status tci_contract_l(tci_context ctx, tci_tensor a, const int32_t* labels_a, tci_tensor b,
                          const int32_t* labels_b, tci_tensor* c, const int32_t* labels_c, int nc);

/* TCI "norm" (Eq. frob_norm): Frobenius norm in FP64 (deterministic
 * two-level reduction).  Synchronises.  Any dtype. */
tci_status tci_norm(tci_context ctx, tci_tensor t, double* out);
/* TCI "normalize" (in place): scale to unit norm; *old_norm (may be NULL)
 * receives the previous norm.  Synchronises. */
tci_status tci_normalize(tci_context ctx, tci_tensor t, double* old_norm);
/* TCI "scale" (in place): t *= (re + i im) (im ignored for real dtypes). */
tci_status tci_scale(tci_context ctx, tci_tensor t, double re, double im);
/* TCI "linear_combine": *out = sum_i coefs[i] ins[i]; coefs are n real
 * values (NULL = all ones).  All inputs share shape and dtype; *out as for
 * tci_contract's c. */
tci_status tci_linear_combine(tci_context ctx, int n, const tci_tensor* ins, const double* coefs,
                              tci_tensor* out);
/* TCI "close" (App. C.2, Miscellaneous): *result = shapes equal and
 * max|a-b| <= eps.  Synchronises. */
tci_status tci_close(tci_context ctx, tci_tensor a, tci_tensor b, double eps, int* result);

/* ------------------------------------------- two-site effective Hamiltonian
 * Textbook two-site DMRG H_eff (the paper names DMRG as a target application
 * in Sec. I; it defines the contraction the matvec is built from):
 *   out[a,s1,s2,b] = sum L[a,wl,a'] W[wl,wm,s1,t1] W[wm,wr,s2,t2]
 *                        R[b,wr,b'] psi[a',t1,t2,b']
 * L: F64 [chiL, Dw, chiL]; R: F64 [chiR, Dw, chiR]; W: F64 [Dw, Dw, d, d]
 * (s = bra/out, t = ket/in); psi, out: F64 [chiL, d, d, chiR]; all
 * row-major contiguous device tensors.  The plan copies what it needs (L, R
 * in the plan's arithmetic, W W pre-contracted), so the caller may free L,
 * W, R after creation.  Arithmetic: the context precision at creation
 * (NATIVE = FP64 everywhere; SPLIT_BF16[_3] = tensor-core contraction,
 * output FP64).
 * Complex plans: L, W, R all C128 (any Dw >= 1, d >= 1; psi and out C128
 * [chiL, d, d, chiR]).  Such a plan applies H_eff as four tci_contract calls
 * in native complex FP64 arithmetic, (psi R) W W L, on copies it owns.
 * tci_heff_apply, tci_heff_flops (8 real flops per complex multiply-add) and
 * tci_lanczos (FP64 vectors; for a Hermitian H_eff, run on its real form:
 * C128 vectors as interleaved FP64 pairs, the real symmetric operator
 * [[Re H, -Im H], [Im H, Re H]] whose spectrum is H's with each eigenvalue
 * twice) accept it; the host-buffer, timed, autotune and config calls return
 * UNSUPPORTED.
 * Errors: SHAPE, DTYPE, ALLOC, CUDA. */
tci_status tci_heff_plan_create(tci_context ctx, tci_tensor L, tci_tensor W, tci_tensor R,
                                tci_heff_plan* plan);
/* Same with a different MPO tensor on each site: W acts on the left site
 * (s1, t1), W2 on the right one (s2, t2), i.e. W W2 in the formula above
 * (non-uniform MPOs).  W2 has W's dtype and shape.  tci_heff_plan_create is
 * this call with W2 = W.  Errors: as tci_heff_plan_create. */
tci_status tci_heff_plan_create2(tci_context ctx, tci_tensor L, tci_tensor W, tci_tensor W2, tci_tensor R,
                                 tci_heff_plan* plan);

/* Replace a real plan's environments (and MPO tensors) by new ones of the
 * same shapes (extension; the paper has no plan object): L [chiL, Dw, chiL],
 * W and W2 [Dw, Dw, 2, 2] (W2 may be NULL: W on both sites), R
 * [chiR, Dw, chiR], row-major F64 device tensors, copied (FP64 plan) or
 * split into bfloat16 pieces (split plans) into the plan's own buffers on the
 * context's stream; the plan's configuration, workspaces and Lanczos graph
 * are kept (the graph is dropped when W.W changes).  A sweep that meets the
 * same bond dimensions again reuses one plan this way.  Errors: INVALID_ARG
 * (invalid plan or tensor handle), DTYPE (a tensor is not F64), SHAPE (not
 * row-major, or shapes differ from the plan's), UNSUPPORTED (complex plans),
 * CUDA. */
tci_status tci_heff_plan_reload(tci_heff_plan plan, tci_tensor L, tci_tensor W, tci_tensor W2, tci_tensor R);
tci_status tci_heff_plan_destroy(tci_heff_plan* plan);
/* out = H_eff psi (async).  psi and out must not overlap. */
tci_status tci_heff_apply(tci_heff_plan plan, tci_tensor psi, tci_tensor out);
/* Same with HOST buffers: psi_host and out_host hold chiL*d*d*chiR doubles;
 * the call copies psi to the device, applies, copies out back and
 * synchronises. */
tci_status tci_heff_apply_host(tci_heff_plan plan, const double* psi_host, double* out_host);
/* tci_heff_apply with CUDA events between its stages, for profiling:
 * stage_ms[0..3] (host) receive the device time of the operand split (0 on
 * the FP64 path), GEMM1 (psi R), the W.W step and GEMM2 (L V).
 * Synchronises. */
tci_status tci_heff_apply_timed(tci_heff_plan plan, tci_tensor psi, tci_tensor out, float* stage_ms);
/* Algorithmic flops of one matvec: 2 chiL d^2 chiR Dw (chiL + chiR) + 2 chiL chiR d^4 Dw^2. */
double tci_heff_flops(tci_heff_plan plan);

/* Allocation-free FP64 H_eff matvec for small bond dimensions.  The paper
 * has no counterpart; it exists for callers that must not allocate device
 * memory when they apply H_eff (a memory manager that owns the whole GPU, a
 * loop where cudaMalloc/cudaFree would synchronise the device, a runtime
 * without an allocator).  Computes the same out = H_eff psi as
 * tci_heff_apply on the FP64 path.  All pointers are device pointers on the
 * current device: L [chiL,5,chiL], W [5,5,2,2], R [chiR,5,chiR], psi and out
 * [chiL,2,2,chiR], row-major, out not overlapping the inputs; work is
 * enqueued on `stream` (a cudaStream_t of the current device, NULL = legacy
 * default stream) and the call returns without waiting.
 * Intermediates live in one fixed 4 MiB device array built into the library
 * (held on every GPU that loads it until exit): requests with
 * 512 + 40*chiL*chiR > 2^19 doubles (chiL*chiR > 13094) are rejected with
 * TCI_ERR_UNSUPPORTED before anything is launched.  All calls share that
 * array, so calls whose kernels overlap on the GPU race; serialise them.  The
 * first call on each device looks up the array's device address (make it
 * before any stream capture).  Allocates no device memory.
 * Errors: INVALID_ARG (NULL pointer, non-positive size), UNSUPPORTED, CUDA;
 * the message is available from tci_last_error(NULL). */
tci_status tci_heff_apply_noalloc(const double* L, const double* W, const double* R, const double* psi,
                                  double* out, int64_t chiL, int64_t chiR, void* stream);

/* TCI "svd" (App. C.2, Tensor linear algebra): a (F64 or F32) is
 * matricised with its first num_of_bds_as_row bonds as the row index
 * (I x J) and factored as U S V^T, s_0 >= ... >= s_{kappa-1} >= 0,
 * kappa = min(I, J).  *u = [d_0..d_{k-1}, kappa], *s = [kappa],
 * *v_dag = [kappa, d_k..d_{r-1}]: new owned tensors of a's dtype (a handle
 * already in *u, *s or *v_dag is freed first).  Computed on the device by
 * one-sided Jacobi in FP64; the singular vectors of zero singular values are
 * zero vectors.  Synchronises.  Errors: INVALID_ARG, SHAPE (k outside
 * 1..order-1), UNSUPPORTED (complex dtype), ALLOC, TIMEOUT (no convergence
 * in 60 sweeps), CUDA. */
tci_status tci_svd(tci_context ctx, tci_tensor a, int num_of_bds_as_row, tci_tensor* u, tci_tensor* s,
                   tci_tensor* v_dag);

/* TCI "trunc_svd" (App. C.2, form (2); form (1) is chi_min = 1,
 * target_trunc_err = 0): as tci_svd, keeping chi singular values chosen by
 * the paper's rules -- (a) drop s_i < s_min; (b) keep at least chi_min, or
 * all that remain after (a) if fewer; (c) add values in descending order
 * until the truncation error sum_{i >= chi} s_i^2 / sum_i s_i^2 <=
 * target_trunc_err or chi = chi_max (chi_max caps chi_min).  *trunc_err
 * (may be NULL) receives that error.  Errors: as tci_svd, and INVALID_ARG
 * when chi_min or chi_max < 1. */
tci_status tci_trunc_svd(tci_context ctx, tci_tensor a, int num_of_bds_as_row, tci_tensor* u, tci_tensor* s,
                         tci_tensor* v_dag, double* trunc_err, int64_t chi_min, int64_t chi_max,
                         double target_trunc_err, double s_min);

/* Two-site finite DMRG (extension; the paper names DMRG as a target of TCI,
 * Sec. I; textbook sweep, Schollwoeck 2011 Secs. 6.2-6.4) for an open chain
 * of nsites sites with the uniform MPO W (device F64 [Dw, Dw, 2, 2], row-major;
 * left boundary vector = its last channel, right boundary = its first), from
 * the Neel product state.  Each bond update: H_eff plan + tci_lanczos
 * (lanczos_steps, started from the current two-site tensor) + tci_trunc_svd
 * (chi_min 1, chi_max, target 0, s_min); the environments follow with
 * tci_contract.  The context's precision applies to every step.
 * energies[nsweeps] (host) receives the last Ritz value of each sweep,
 * max_trunc_err[nsweeps] (host, may be NULL) the largest truncation error of
 * each sweep.  Synchronises.  Errors: SHAPE, INVALID_ARG, and those of the
 * calls it makes. */
tci_status tci_dmrg(tci_context ctx, tci_tensor W, int nsites, int64_t chi_max, int nsweeps, int lanczos_steps,
                    double s_min, double* energies, double* max_trunc_err);

/* iTEBD ground-state iteration of the paper's App. A (extension: the
 * application of Sec. III A as one call).  h: device F64 two-site term
 * h[(s1 s2), (t1 t2)] ([4, 4] or [2, 2, 2, 2], row-major); the gate
 * u = exp(-dt h) is formed on the device.  gamma_a, gamma_b [chi_l, 2, chi_r]
 * and lambda_a, lambda_b [chi] (device F64, row-major) are the two-site unit
 * cell; they are updated in place (their storage is replaced by arrays the
 * handles then own, with the bond dimensions the truncation chose).  Each of
 * niters iterations forms Theta = L_B Gamma_A L_A Gamma_B L_B, applies u,
 * truncates with tci_trunc_svd (chi_min 1, chi, target 0, s_min), normalises
 * Lambda_A and re-gauges with 1/Lambda_B, alternating A and B.  energies[i]
 * (host) = -log ||Theta'||^2 / (2 dt), the energy per site estimate;
 * trunc_errs[i] (host, may be NULL) the truncation error.  Synchronises.
 * Errors: SHAPE, INVALID_ARG, and those of the calls it makes. */
tci_status tci_itebd(tci_context ctx, tci_tensor h, double dt, tci_tensor gamma_a, tci_tensor gamma_b,
                     tci_tensor lambda_a, tci_tensor lambda_b, int64_t chi, double s_min, int niters,
                     double* energies, double* trunc_errs);

/* Belief propagation on the norm network of a tensor-network state (App. B;
 * extension: the message iteration as one call).  Graph: nsites vertices and
 * nedges edges (host int64 pairs edges[2e], edges[2e + 1], distinct
 * vertices).  sites[i] (device F64, row-major) is V_i[s, b_1 .. b_k]: the
 * physical bond first, then one bond per neighbour in ascending neighbour
 * order (k = degree of i, at most 6).  messages[2e] is the message u -> v of
 * edge e = (u, v), messages[2e + 1] the message v -> u; each is an F64
 * [chi_e, chi_e] matrix (ket bond index, bra bond index), updated in place.
 * One iteration replaces every message, from the previous set, by
 *   M_{i->j}[b, b'] = sum V_i[s, .., b, ..] V_i[s, .., b', ..] prod_{k != j} M_{k->i}
 * normalised to unit Frobenius norm.  Messages with the same site shape and
 * outgoing bond run as one batched contraction.  Iterations stop after
 * niters or once the residual max_m ||M_new - M_old||_F is <= tol;
 * residuals[it] (host, may be NULL; niters entries) and *iters_done (may be
 * NULL) report them.  Synchronises.  Errors: INVALID_ARG, SHAPE, DTYPE and
 * those of the calls it makes. */
tci_status tci_bp(tci_context ctx, int nsites, int nedges, const int64_t* edges, const tci_tensor* sites,
                  tci_tensor* messages, int niters, double tol, int* iters_done, double* residuals);

/* Vector arithmetic of tci_lanczos (extension; the paper has no Lanczos
 * API).  TCI_LANCZOS_F64: vectors in FP64, every dot product and every
 * update term that is not at rounding level in FP64 (rounding-level
 * Gram-Schmidt terms are summed in FP32 under an error bound below FP64
 * rounding, see tci_heff_lanczos_stats).
 * TCI_LANCZOS_DF32: vectors held as pairs of FP32 numbers hi + lo
 * (double-float, Dekker 1971; ~48 significant bits) with error-free
 * transformations, so the vector passes run on the FP32 pipes (B300 issues
 * FP64 FMAs at ~1/64 of its FP32 rate); Ritz values agree with the FP64
 * arithmetic to ~1e-10 relative or better.  TCI_LANCZOS_AUTO (default):
 * FP64. */
typedef enum {
  TCI_LANCZOS_AUTO = 0,
  TCI_LANCZOS_F64 = 1,
  TCI_LANCZOS_DF32 = 2
} tci_lanczos_arith;

/* Select the vector arithmetic of later tci_lanczos calls on `plan`.
 * Errors: INVALID_ARG (invalid plan or value), INVALID_CONTEXT. */
tci_status tci_heff_set_lanczos_arith(tci_heff_plan plan, tci_lanczos_arith arith);

/* Re-orthogonalisation of tci_lanczos (extension).  Every step projects
 * H v_j against the whole basis by classical Gram-Schmidt.
 * TCI_GS_DGKS (default): the projection is repeated only where the first
 * one cancelled, ||w'|| < ||w|| / sqrt(2) (Daniel, Gragg, Kaufman & Stewart,
 * Math. Comp. 30, 1976); where it is not repeated the second projection
 * would change w only at rounding level.  TCI_GS_TWICE: always twice (CGS2).
 * Errors: INVALID_ARG (invalid plan or value), INVALID_CONTEXT. */
typedef enum {
  TCI_GS_DGKS = 0,
  TCI_GS_TWICE = 1
} tci_gram_schmidt;
tci_status tci_heff_set_gram_schmidt(tci_heff_plan plan, tci_gram_schmidt mode);

/* Lanczos ground state of H_eff (textbook; Golub & Van Loan Sec. 10.1 with
 * full classical Gram-Schmidt re-orthogonalisation when reorth != 0, see
 * tci_heff_set_gram_schmidt; Ritz value by Sturm bisection, Sec. 8.4).  All vector work runs on the device, in the
 * arithmetic chosen by tci_heff_set_lanczos_arith (FP64 by default);
 * scalars (alpha, beta, Gram-Schmidt coefficients, the tridiagonal
 * eigenpair) are FP64.
 * psi0: start vector [chiL,d,d,chiR] F64 (normalised internally, not
 * modified).  Runs up to nsteps (1..256) steps, stopping early when
 * beta_j < 1e-12 |alpha_j|.  Outputs (host): *ritz, alpha[nsteps],
 * beta[nsteps] (entries past *steps_done are 0), *steps_done.  x (may be
 * NULL): device F64 tensor shaped like psi0 receiving the unit Ritz vector.
 * Synchronises.  Errors: INVALID_ARG, SHAPE, ALLOC, CUDA. */
tci_status tci_lanczos(tci_heff_plan plan, tci_tensor psi0, int nsteps, int reorth, double* ritz,
                       double* alpha, double* beta, int* steps_done, tci_tensor x);

/* Counters of the last tci_lanczos on `plan` (extension), into stats[5]
 * (host): [0] steps done; [1] steps whose Gram-Schmidt projection was
 * repeated (DGKS) or, with TCI_GS_TWICE, every re-orthogonalised step;
 * [2] update passes whose rounding-level terms (coefficients of v_0 ..
 * v_{j-2}, 1-norm at most 2^-32 ||w|| / (k + 8) for k such terms) were
 * summed in FP32 and subtracted in FP64, adding an error below 2^-56 ||w||;
 * [3] update passes whose small terms (1-norm at most 2^-10 ||w|| / (k + 8),
 * k >= 6; e.g. the matvec-error-level terms of a split-precision plan) were
 * summed in double-float arithmetic under the same error bound; [4] steps
 * whose second projection was applied in FP32 and folded into the
 * next-vector pass with beta_j^2 = ||w'||^2 - |h'|^2.  [2] to [4] stay 0
 * for double-float vectors, without re-orthogonalisation, with reduced terms
 * switched off (tci_heff_set_lanczos_reduced_terms) and on steps whose vector
 * work runs as one cluster launch (n (j + 2) <= 2^19); [2] and [3] also for
 * vectors shorter than 2^20 elements and bases beyond 20 vectors.  All zero
 * before the first solve.  Errors: INVALID_ARG, INVALID_CONTEXT. */
tci_status tci_heff_lanczos_stats(tci_heff_plan plan, int* stats);

/* First Gram-Schmidt projection of tci_lanczos formed inside the matvec
 * (extension; off by default): on split-BF16 plans with FP64 vectors the dot
 * products <v_i, H v_j> (i <= j, basis up to 23 vectors) and ||H v_j||^2 are
 * computed in FP64 by the epilogue of the matvec's second GEMM from the
 * output tiles it stores, instead of a separate pass over the basis; per-CTA
 * partial sums are added in a fixed order.  Results agree with the separate
 * pass to FP64 rounding.  On B300 it is slower (measured at chi = 2048: the
 * GEMM takes 2.0 / 2.9 / 4.5 ms with 1 / 10 / 20 basis vectors against 1.55 ms
 * plus 0.1-0.6 ms for the separate pass), because the epilogue threads'
 * extra state spills registers and their dot products wait on DRAM between
 * accumulator drains.  Errors: INVALID_ARG, INVALID_CONTEXT. */
tci_status tci_heff_set_lanczos_fused_dots(tci_heff_plan plan, int enable);

/* Double-float Gram-Schmidt dot products in tci_lanczos (extension; off by
 * default: every Lanczos dot product is FP64).  On split-BF16 plans with FP64
 * vectors and re-orthogonalisation, enable = 1 stores each basis vector v_i
 * also as an FP32 pair hi + lo (|v_i - hi - lo| <= 2^-47 |v_i| per element,
 * hi and lo in separate planes), written by the pass that writes v_i; the
 * first projection's dot products <v_i, w> and ||w||^2 are then summed from
 * that copy in double-float arithmetic (products made exact with FMA, Knuth
 * sums) on the FP32 pipes, and the second projection's dots (formed in the
 * update pass whose small terms are double-float) from FP32 pairs split on the
 * integer pipes; both passes become bound by HBM instead of B300's FP64 rate,
 * and the pass-3 correction reads the copy's hi planes.  Each dot product
 * agrees with the FP64 one to about 1e-14 ||v_i|| ||w||, above FP64
 * rounding; the update passes and the recurrence scalars stay FP64.  The copy
 * takes 8 bytes per basis element of device memory (without this option a
 * split plan keeps the hi planes only, 4 bytes per element, which the pass-3
 * correction reads).  Ignored when
 * tci_heff_set_lanczos_fused_dots is on.  Errors: INVALID_ARG, INVALID_CONTEXT. */
tci_status tci_heff_set_lanczos_shadow_dots(tci_heff_plan plan, int enable);

/* Reduced-precision small update terms of tci_lanczos with FP64 vectors
 * (extension; on by default): the FP32 and double-float evaluations of
 * rounding-level and matvec-error-level Gram-Schmidt terms counted by
 * tci_heff_lanczos_stats [2] to [4], each under an added error below
 * 2^-56 ||w||.  enable = 0 keeps every update term in FP64 (slower on B300,
 * equal to rounding).  Errors: INVALID_ARG, INVALID_CONTEXT. */
tci_status tci_heff_set_lanczos_reduced_terms(tci_heff_plan plan, int enable);

/* CUDA-graph replay of tci_lanczos on real plans (extension; on by
 * default).  A solve launches a sequence fixed by its
 * arguments (whether x is given, nsteps, reorth, the vector arithmetic,
 * the Gram-Schmidt mode and the plan's GEMM configuration), every branch
 * being decided on the device; the first call with a given sequence runs
 * eagerly, the second captures it into a graph and later calls replay the
 * graph (with the call's psi0 and x addresses), so the host enqueues one
 * launch per solve.  enable = 0 runs every solve eagerly and releases the
 * graph.  Results are identical either way.
 * Errors: INVALID_ARG, INVALID_CONTEXT. */
tci_status tci_heff_set_lanczos_graphs(tci_heff_plan plan, int enable);

/* Graph replay state of `plan` (extension): info[0] = 1 while replay is
 * enabled (a failed capture turns it off and later solves run eagerly),
 * info[1] = 1 when the last tci_lanczos ran as one graph launch and 0 when it
 * ran eagerly, info[2] = graph launches of this plan so far.  info holds 3
 * int64_t.  Errors: INVALID_ARG (invalid plan, NULL info), INVALID_CONTEXT. */
tci_status tci_heff_lanczos_graph_info(tci_heff_plan plan, int64_t* info);

/* ------------------------------------------- U(1) block-sparse H_eff
 * Charge-conserving (U(1)) block-sparse tensors are listed as future work of
 * TCI (Sec. IV); the operation is the two-site H_eff above applied to the
 * zero-filled tensors, computed block by block over the charge-allowed
 * blocks only.  Charges: sector_charge[nsec] (distinct; bond sector i has
 * dimension sector_dim[i]), phys_charge[2] of the physical states,
 * mpo_charge[5] of the MPO channels (W[wl,wr,s,t] != 0 only if
 * phys_charge[s]-phys_charge[t] = mpo_charge[wl]-mpo_charge[wr]).  These four
 * arrays are HOST pointers.
 * Packed layouts (device, FP32, each block row-major, blocks back to back):
 *   psi/out: blocks (ia, t1, t2, ib) for ia = 0.., t1 = 0..1, t2 = 0..1 in
 *            that nesting order, present iff q_ib = q_ia + c(t1) + c(t2);
 *            block shape [dim ia, dim ib];
 *   L, R:    blocks (i, w, j) for i = 0.., w = 0..4, present iff
 *            q_j = q_i + Delta(w); block shape [dim i, dim j]
 * (q = sector_charge, c = phys_charge, Delta = mpo_charge).  W is the dense
 * device F64 MPO [5,5,2,2].  The plan packs L and R into the tensor-core
 * operand layout once, so the caller may free them after creation.
 * Arithmetic: the context precision (must be SPLIT_BF16 or SPLIT_BF16_3).
 * Every block GEMM of one matvec stage runs in a single grouped persistent
 * launch, the blocks that share a sector stacked into one GEMM problem.
 * Errors: INVALID_ARG, UNSUPPORTED (NATIVE precision, or sector blocks whose
 * offsets exceed 32 bits in the W.W step: a sector dimension times five sector
 * dimensions beyond 2^31), ALLOC, CUDA. */
tci_status tci_bs_heff_plan_create(tci_context ctx, int nsec, const int32_t* sector_charge,
                                   const int64_t* sector_dim, const int32_t* phys_charge,
                                   const int32_t* mpo_charge, const float* L_packed,
                                   const float* R_packed, const double* W, tci_bs_plan* plan);
tci_status tci_bs_plan_destroy(tci_bs_plan* plan);
/* out = H_eff psi on packed block-sparse vectors (device FP32, length
 * tci_bs_psi_size).  Async on the context stream; psi and out must not
 * overlap. */
tci_status tci_bs_heff_apply(tci_bs_plan plan, const float* psi, float* out);
/* Algorithmic flops of one matvec: 2 m n k over every charge-allowed block
 * product of both GEMM stages plus 2 d^4 Dw^2 per element of every sector
 * pair that carries an intermediate block.  -1/0 for an invalid plan. */
double tci_bs_heff_flops(tci_bs_plan plan);
int64_t tci_bs_psi_size(tci_bs_plan plan);
/* Profiling form of tci_bs_heff_apply: stage_ms[0..3] (host) receive the
 * device times of the psi split, grouped GEMM1, W.W tasks and grouped GEMM2
 * (with the unpack of its staged result into the packed output blocks).
 * Synchronises. */
tci_status tci_bs_heff_apply_timed(tci_bs_plan plan, const float* psi, float* out, float* stage_ms);
/* BF16 tensor-core flops the two grouped launches execute per matvec
 * (2 x products x M N Kp summed over block GEMMs). */
double tci_bs_tensor_flops(tci_bs_plan plan);

/* ------------------------------------------- batched TEBD theta
 * The theta formation and gate application of the paper's iTEBD listing
 * (App. A), batched over independent bonds:
 *   theta_i[a,s1,s2,b] = sum_{t1,t2,c} G_i[s1,s2,t1,t2] A_i[a,t1,c] B_i[c,t2,b]
 * (G's LAST two indices are summed; the listing's "ijkl","jkmn"->"imnl" sums
 * the gate's FIRST two -- the two agree for symmetric gates.)  complex64,
 * d = 2.  chi[nbonds] is a HOST array of bond dimensions.  Packed device
 * layouts (interleaved re/im, bonds back to back, each row-major):
 * A_i [chi_i,2,chi_i], B_i [chi_i,2,chi_i], G_i [2,2,2,2] (16 values per
 * bond), theta_i [chi_i,2,2,chi_i]; A, B, theta 8-byte and G 16-byte
 * aligned (else INVALID_ARG).  Arithmetic: the context precision at
 * plan creation (SPLIT_BF16 or SPLIT_BF16_3): the complex product is one
 * real split-BF16 tensor-core GEMM per bond ([Ar | Ai] times [Br | -Bi] and
 * [Bi | Br], real and imaginary parts in adjacent output columns), all bonds
 * in one grouped persistent launch whose epilogue applies the gate (AB is
 * never stored).  Errors: INVALID_ARG, UNSUPPORTED (NATIVE precision),
 * ALLOC, CUDA. */
tci_status tci_tebd_plan_create(tci_context ctx, int nbonds, const int64_t* chi, tci_tebd_plan* plan);
tci_status tci_tebd_plan_destroy(tci_tebd_plan* plan);
/* theta = batched theta(A, B, G); async on the context stream. */
tci_status tci_tebd_apply(tci_tebd_plan plan, const void* A, const void* B, const void* G, void* theta);
/* Algorithmic flops: sum_i 8 chi_i^3 d^2 + 8 chi_i^2 d^4 (8 real flops per complex multiply-add). */
double tci_tebd_flops(tci_tebd_plan plan);
/* The same batch on tensor handles (one call, no plan kept): A[i], B[i]
 * C64 row-major [chi_i, 2, chi_i], G[i] C64 [2, 2, 2, 2]; theta[i] C64
 * [chi_i, 2, 2, chi_i] (written), or NULL handles, which receive new owned
 * tensors.  Builds a plan for these chi_i, packs the operands with device
 * copies, applies it and unpacks theta; synchronises.  Arithmetic as
 * tci_tebd_plan_create (the context precision; NATIVE is UNSUPPORTED).
 * Errors: INVALID_ARG, DTYPE, SHAPE, UNSUPPORTED, ALLOC, CUDA. */
tci_status tci_tebd_theta_batched(tci_context ctx, int n, const tci_tensor* A, const tci_tensor* B,
                                  const tci_tensor* G, tci_tensor* theta);
/* Profiling form of tci_tebd_apply: stage_ms[0..2] (host) receive the device
 * times of the split and of the grouped GEMM (whose epilogue applies the
 * gate), and 0 (there is no separate gate stage).  Synchronises. */
tci_status tci_tebd_apply_timed(tci_tebd_plan plan, const void* A, const void* B, const void* G, void* theta,
                                float* stage_ms);
/* BF16 tensor-core flops the grouped launch executes (one real GEMM per bond,
 * M = 2 chi, N = 4 chi, K = 2 pad8(chi)). */
double tci_tebd_tensor_flops(tci_tebd_plan plan);

/* ------------------------------------------- autotuner and plan cache
 * (An implementation facility; the paper has no counterpart.)  Time the
 * candidate configurations of the split-BF16 tensor-core GEMM on the plan's
 * own operands -- the hi*hi accumulation chunk (128/256/512, capped by
 * max_chunk_k: the measured relative error of the chi = 2048 matvec is
 * 2.2e-7 / 4.3e-7 / 8.8e-7), the cross-product chunk (1024/4096) and the
 * tile order (m-fastest or groups of 8/16 m-blocks) -- and keep the fastest
 * in the plan: the candidates first run in turn for at least 250 ms (the clock
 * settles under the power cap), then each keeps the median of four timed
 * rounds, and near ties (2 %) go to the grouped tile order (16, then 8), the
 * longer chunks and the wider tile.  Results are cached per (plan kind, shape, device) in memory
 * and, when TCI_AUTOTUNE_CACHE names a file, in that file (read first, so a
 * cached shape is not timed again); the W.W kernel variant is timed too
 * (not cached).  chosen (may be NULL) receives 3 ints: chunk_k, xchunk_k,
 * raster.  The inputs are used as timing data only
 * (outputs are overwritten).  Synchronises.  Errors: INVALID_ARG, SHAPE, CUDA. */
tci_status tci_heff_autotune(tci_heff_plan plan, tci_tensor psi, tci_tensor out, int max_chunk_k, int* chosen);
/* Read / set the configuration of a split-BF16 H_eff plan (extension; no
 * counterpart in the paper): cfg[0] chunk_k, cfg[1] xchunk_k (as in
 * tci_context_set_split_chunks), cfg[2] raster (tile order: 0 m-fastest,
 * G > 0 groups of G m-blocks), cfg[3] a' per thread of the W.W kernel
 * (2 or 4).  tci_heff_autotune sets all four; set_config lets a caller
 * replay a known configuration without timing.  For an FP64 plan get
 * returns zeros and set is rejected.  Errors: INVALID_ARG (invalid plan,
 * NULL cfg, values outside the rules above), UNSUPPORTED (FP64 plan). */
tci_status tci_heff_get_config(tci_heff_plan plan, int* cfg);
tci_status tci_heff_set_config(tci_heff_plan plan, const int* cfg);
/* The same for block-sparse and TEBD plans, whose grouped launches also try
 * the tile shape: 128 x 128 or 128 x 64 output tiles (narrow tiles carry
 * less padding and half the MMA work on problems of few columns); the
 * chosen width is read with tci_bs_tile_n / tci_tebd_tile_n.  chosen as
 * above (3 ints). */
tci_status tci_bs_autotune(tci_bs_plan plan, const float* psi, int max_chunk_k, int* chosen);
tci_status tci_tebd_autotune(tci_tebd_plan plan, const void* A, const void* B, const void* G, void* theta,
                             int max_chunk_k, int* chosen);
/* Tile width (output columns per tile, 64 or 128) of a block-sparse or TEBD
 * plan's grouped GEMMs: set it (a captured graph is dropped and re-captured
 * by the next apply) or read it (-1 for an invalid plan).  Set errors:
 * INVALID_ARG (invalid plan, width not 64 or 128), INVALID_CONTEXT. */
tci_status tci_bs_set_tile_n(tci_bs_plan plan, int bn);
int tci_bs_tile_n(tci_bs_plan plan);
tci_status tci_tebd_set_tile_n(tci_tebd_plan plan, int bn);
int tci_tebd_tile_n(tci_tebd_plan plan);
/* W.W pass of a block-sparse plan (the W.W coefficients applied to GEMM1's
 * outputs, written as GEMM2's bf16 pieces): variant 0 stages 32 a' x 8 b
 * tiles in shared memory, one output pair per thread; variants 1, 2, 3 give
 * each thread a 4 a' x 4 b micro-tile, read as 16-byte rows and written as
 * 8-byte piece vectors without shared memory, for all 20 outputs (1), or for
 * a quarter (2) or a tenth (3) of them.  All form every element with the
 * same terms in the same order, so the results agree bit for bit;
 * tci_bs_autotune times them inside the matvec sequence.  Set (a captured
 * graph is dropped and re-captured by the next apply) or read it (-1 for an
 * invalid plan).  Set errors: INVALID_ARG (invalid plan, variant not in
 * 0..3), INVALID_CONTEXT. */
tci_status tci_bs_set_ww_variant(tci_bs_plan plan, int variant);
int tci_bs_ww_variant(tci_bs_plan plan);

#ifdef __cplusplus
}
#endif
#endif /* TCI_B300_H */
