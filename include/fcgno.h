/*
 * fcgno.h - C ABI of the GB300 FCG-NO library.
 *
 * The library runs the flexible conjugate gradient method of Algorithm 1 (Section 2.3 of
 * Rudikov et al., "Neural operators meet conjugate gradients: the FCG-NO method",
 * arXiv 2402.05598), preconditioned by a Fourier neural operator (Section 2.4.2,
 * Appendix A), on the 5-point finite-volume discretisation of -div(k grad u) = f on the
 * unit square with zero Dirichlet data (Eq. (1)-(2)).
 *
 * Conventions shared by every call
 *  - Grid: N x N interior nodes, h = 1/(N+1), node (p, q) at ((p+1)h, (q+1)h). A field is
 *    a contiguous row-major double array [N][N] indexed [q][p] (p fastest); a batch of B
 *    instances is [B][N][N]. Face coefficients are harmonic means of neighbouring k, a
 *    boundary face takes the k of its node; the operator includes the 1/h^2 factor.
 *  - Pointers are DEVICE pointers owned by the caller unless a parameter says "host".
 *    The library never frees caller memory. Handles (fcgno_op_t, fcgno_model_t) are owned
 *    by the library and released with their destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls are
 *    asynchronous on that stream except where stated.
 *  - No C++ exception crosses this boundary. Argument errors return FCGNO_EINVAL before
 *    any launch; CUDA failures return FCGNO_ECUDA (fcgno_last_error() gives the text).
 *  - Per-instance solve outcomes are reported in fcgno_solve_info[b].status.
 *  - The tensor-core kernels bound every wait on an on-chip barrier (about 1 s); one that
 *    gives up sets its operator's error flag and returns. fcgno_solve and fcgno_bucket_poll
 *    read and clear that flag after their own synchronisation and then return FCGNO_ETIMEOUT
 *    (the results of that call are invalid); a timeout inside the asynchronous
 *    fcgno_precond_apply or a FCGNO_BF16 fcgno_train_step is reported by the next
 *    fcgno_solve or fcgno_bucket_poll on the same operator.
 *  - Every computation runs in CUDA kernels of this library (sm_103a); there is no host
 *    fallback.
 *  - Concurrency: calls on different operators may run on different streams at the same
 *    time, also with one shared model, when the preconditioner is FCGNO_BF16 or FCGNO_FP16
 *    (its activations belong to the operator). The FCGNO_FP64 / FCGNO_FP32 preconditioner and
 *    fcgno_train_step keep their activations in the model: calls using them on one model
 *    must not overlap. Calls on one operator must not overlap either. Changing a model's
 *    weights (fcgno_model_sync) while a solve or bucket uses it is not supported.
 *    Host threads: the library's global state (last error, launch counter, tracing) is
 *    thread-safe, but a model builds its 16-bit weight images and transform tables on its
 *    first use for each precision and grid size; that first use must not run concurrently
 *    with another host thread's call on the same model (issue it once, or serialise the
 *    calls, before sharing the model across threads).
 */
#ifndef FCGNO_H
#define FCGNO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FCGNO_OK = 0,
  FCGNO_EINVAL = 1,     /* bad argument (checked before any launch)                      */
  FCGNO_ENOMEM = 2,     /* device allocation failed                                        */
  FCGNO_ECUDA = 3,      /* a CUDA call or kernel failed                                    */
  FCGNO_ENOCONV = 4,    /* instance status: max_iter reached before tol                    */
  FCGNO_EBREAKDOWN = 5, /* instance status: (p_i, s_i) zero or non-finite (Algorithm 1)    */
  FCGNO_ETIMEOUT = 6    /* a bounded device wait gave up (kernel returned an error flag)   */
} fcgno_status;

typedef enum {
  FCGNO_FP64 = 0, /* preconditioner computed in FP64 on CUDA cores                         */
  FCGNO_BF16 = 1, /* preconditioner GEMMs in BF16 on tcgen05 tensor cores, FP32 accumulate */
  FCGNO_FP16 = 2, /* as BF16 with FP16 operands                                            */
  FCGNO_FP32 = 3  /* preconditioner computed in FP32 on CUDA cores                         */
} fcgno_prec;

typedef struct fcgno_op* fcgno_op_t;
typedef struct fcgno_model* fcgno_model_t;

/* Shape of the Fourier neural operator (Appendix A: encoder, `layers` Fourier layers,
 * decoder). modes = M keeps x1-frequencies 0..M-1 and -M..-1 and x2-frequencies 0..M-1;
 * requires N >= 2M for every grid it is applied to. in_channels must be 2.
 * output_scale chooses how the decoder's output is put back into the units of A^-1 (the
 * paper leaves the network's scaling open): 0 multiplies it by h^2 rms(r); 1 also divides it,
 * grid point by grid point, by the coefficient k (z = h^2 rms(r) NO(...) / k), so that the
 * contrast of k, which the network would otherwise have to reproduce through its GELUs,
 * enters the way it enters A^-1 at the highest frequencies (about h^2 r / (4 k)). */
typedef struct {
  int width;        /* C   */
  int layers;       /* L   */
  int modes;        /* M   */
  int proj_width;   /* C_p */
  int in_channels;  /* 2: (r / rms(r), log k) */
  int output_scale; /* 0: h^2 rms(r); 1: h^2 rms(r) / k */
} fcgno_model_desc;

typedef struct {
  double tol;      /* stop instance b when ||r_i|| <= tol * ||r_0|| (Table 1 criterion)    */
  int m_max;       /* truncation m_max of Algorithm 1, 1 <= m_max <= 8                       */
  int max_iter;    /* iteration cap                                                          */
  int fixed_iters; /* nonzero: ignore tol and run exactly max_iter iterations                */
  int check_every; /* host reads the convergence counter every this many iterations (>=1); */
                   /* once 32 or fewer instances run, every min(check_every, 2) iterations   */
} fcgno_solve_opts;

typedef struct {
  int32_t iters;   /* iterations performed                                                   */
  int32_t status;  /* FCGNO_OK (converged), FCGNO_ENOCONV or FCGNO_EBREAKDOWN                */
  double relres;   /* ||r_iters|| / ||r_0|| on the recursively updated residual              */
  double r0norm;   /* ||r_0||                                                                */
} fcgno_solve_info;

/* Stencil assembly (Eq. (1)-(2)): k is [batch][N][N] (k > 0). Builds the face
 * coefficients and log k on the device and returns a handle that owns them.
 * Errors: EINVAL if N < 2, batch < 1, k or out NULL; ENOMEM; ECUDA. */
fcgno_status fcgno_assemble(int N, int batch, const double* k, void* stream, fcgno_op_t* out);
/* Re-assembles an existing operator in place from new coefficient fields k ([batch][N][N]
 * with the operator's N and batch; k > 0): same arithmetic as fcgno_assemble, no allocation,
 * asynchronous on `stream`. The operator's solver workspace, captured graphs and 16-bit
 * activations stay valid, so a batch of new problems of the same shape reuses them.
 * Errors: EINVAL for a NULL op or k; ECUDA. */
fcgno_status fcgno_reassemble(fcgno_op_t op, const double* k, void* stream);
/* Releases the handle and everything it owns (solver workspace, graphs, the 16-bit
 * preconditioner's activations) with cudaFree, which waits for work in flight on the
 * device. NULL is a no-op. */
fcgno_status fcgno_op_destroy(fcgno_op_t op);
/* y = A x for every instance (x, y: [batch][N][N], may not alias).
 * Errors: EINVAL for a NULL op, x or y, or x == y. */
fcgno_status fcgno_apply_A(fcgno_op_t op, const double* x, double* y, void* stream);
/* Training pairs for residuals that are not Krylov vectors (the random-residual ablation of
 * Section 3.5, Eq. (11) in error form): r_out = b - A u and e_out = u_star - u for every
 * instance (all [batch][N][N], device; u_star solves A u_star = b). Asynchronous.
 * Errors: EINVAL for a NULL argument or r_out / e_out aliasing u. */
fcgno_status fcgno_residual_pair(fcgno_op_t op, const double* b, const double* u, const double* u_star,
                                 double* r_out, double* e_out, void* stream);

/* Neural operator handle. `weights` is a DEVICE float32 blob of fcgno_weight_count(desc)
 * elements in this order (row-major): lift_w [C][2], lift_b [C]; per layer l: w_l [C][C]
 * (out, in), b_l [C], r_l [2M][M][C][C][2] (x1-mode slot j -> frequency j or j-2M, x2-mode,
 * in, out, re/im); proj1_w [Cp][C], proj1_b [Cp], proj2_w [Cp], proj2_b [1].
 * The handle keeps the pointer (caller keeps the blob alive) and derives reduced-precision
 * copies from it; call fcgno_model_sync after the blob changes.
 * fcgno_weight_count returns 0 for an invalid desc. create: EINVAL for a NULL desc, weights
 * or out, width or proj_width outside 1..64, layers outside 1..16, modes outside 1..16, or
 * in_channels != 2; ENOMEM. Shapes the 16-bit path does not support (it needs width 16 or
 * 32, proj_width = width, N = 32, 64 or a multiple of 128) make fcgno_precond_apply,
 * fcgno_solve, fcgno_solve_host and fcgno_bucket_create return EINVAL for FCGNO_BF16 /
 * FCGNO_FP16, before any launch.
 * sync: EINVAL for a NULL model. destroy: NULL is a no-op. */
size_t fcgno_weight_count(const fcgno_model_desc* desc);
fcgno_status fcgno_model_create(const fcgno_model_desc* desc, const float* weights, void* stream,
                                fcgno_model_t* out);
fcgno_status fcgno_model_sync(fcgno_model_t model, void* stream);
fcgno_status fcgno_model_destroy(fcgno_model_t model);

/* z = NO(r, log k) for every instance of op (Algorithm 1, w_i = B(r_i); Appendix A):
 * z = s * decoder(Fourier layers(encoder(r / rms(r), log k))), z = 0 where r = 0, with
 * s = h^2 rms(r) (output_scale 0) or h^2 rms(r) / k at each grid point (output_scale 1)
 * (h = 1/(N+1); the h^2 factor gives the output the units of A^-1).
 * r, z: [batch][N][N]. prec selects the arithmetic (FP64, FP32, BF16, FP16).
 * Errors: EINVAL for a NULL argument, N < 2*modes, an unknown precision or a shape the
 * 16-bit path does not support (all before any launch); ENOMEM; ECUDA. */
fcgno_status fcgno_precond_apply(fcgno_model_t model, fcgno_op_t op, const double* r, double* z,
                                 fcgno_prec prec, void* stream);

/* Algorithm 1 for every instance of A: x holds u_0 on entry and the iterate on exit;
 * b is [batch][N][N]; Bpc NULL runs the identity preconditioner (plain CG for m_max = 1).
 * info is a HOST array of batch entries. Synchronises on `stream` every check_every
 * iterations (every min(check_every, 2) once 32 or fewer instances run) and at exit (the
 * call returns when every instance has stopped).
 * Errors: EINVAL for a NULL A, b or x, bad opts (tol < 0, m_max outside 1..8,
 * max_iter < 0), N < 2*modes, an unknown precision or a shape the 16-bit path does not
 * support; ENOMEM; ECUDA; ETIMEOUT (see the
 * conventions). Per-instance outcomes (converged, not converged, breakdown) are in info. */
fcgno_status fcgno_solve(fcgno_op_t A, fcgno_model_t Bpc, const double* b, double* x,
                         const fcgno_solve_opts* opts, fcgno_prec prec, fcgno_solve_info* info,
                         void* stream);

/* Algorithm 1 preconditioned by Jacobi(steps) (Eq. (15); the Jacobi column of Table 1):
 * w_i = x_steps with x_0 = 0, x_{j+1} = x_j + D(A)^-1 (r_i - A x_j), FP64. The classical
 * baseline the paper compares the neural preconditioner against. Same arguments and
 * results as fcgno_solve; EINVAL for steps outside 1..64. */
fcgno_status fcgno_solve_jacobi(fcgno_op_t A, int steps, const double* b, double* x, const fcgno_solve_opts* opts,
                                fcgno_solve_info* info, void* stream);

/* End-to-end variant of fcgno_solve on HOST buffers: k_host, b_host, x_host are
 * [batch][N][N] host arrays (pinned memory gives the fastest copies). Copies k, b, x in,
 * assembles, solves, copies x out; info is a host array. Synchronous.
 * The device copies of k, b, x and the assembled operator (with its Krylov workspace and
 * captured graphs) of the last 4 shapes (device, N, batch) are kept for the next call of the
 * same shape, which then re-assembles in place (fcgno_reassemble); fcgno_solve_host_release
 * frees them. A call whose shape is being solved by another thread uses temporary buffers.
 * Errors: EINVAL for N < 2, batch < 1 or a NULL host buffer, then those of fcgno_solve. */
fcgno_status fcgno_solve_host(int N, int batch, const double* k_host, const double* b_host,
                              double* x_host, fcgno_model_t Bpc, const fcgno_solve_opts* opts,
                              fcgno_prec prec, fcgno_solve_info* info, void* stream);
/* Frees the device state fcgno_solve_host keeps between calls (waits for work in flight). */
fcgno_status fcgno_solve_host_release(void);

/* Allocation-free variant of fcgno_solve for the identity preconditioner (B = I; plain CG
 * for m_max = 1). The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they solve, e.g. code that runs under a fixed,
 * pre-reserved memory budget or in a context where the CUDA allocator must not be entered.
 * It calls no cudaMalloc/cudaFree and no allocating library routine; its Krylov state
 * (r, the m_max+1 directions p_k and s_k, per-instance scalars and partial sums) lives in
 * one file-scope device array of 8 MiB that every GPU loading the library keeps until the
 * process exits. Problems whose state does not fit (about 8*N*N*batch*(2*m_max+3) bytes
 * plus small terms) are rejected with FCGNO_EINVAL and a message giving the size needed.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and keeps it for the life of the process; make that first call before any stream capture.
 * A cudaDeviceReset invalidates that address together with every handle of this library:
 * use none of them afterwards. Every call shares the array and leaves
 * its contents behind, so two calls that overlap on the GPU (different streams, threads
 * or processes sharing the context) race and corrupt each other. Arguments and results
 * are those of fcgno_solve with Bpc = NULL and prec = FCGNO_FP64; info is a HOST array. */
fcgno_status fcgno_solve_noalloc(fcgno_op_t A, const double* b, double* x, const fcgno_solve_opts* opts,
                                 fcgno_solve_info* info, void* stream);

/* Krylov-subspace sampling (Eq. (9), Section 3.1): runs K iterations of CG (Algorithm 1
 * with B = I, m_max = 1) from x0 on every instance and stores, for i = 1..K, the
 * residual r_i and the error e_i = u_star - u_i:
 * r_out, e_out are [K][batch][N][N]; u_star is [batch][N][N] (the converged solution).
 * Rows after an instance has converged repeat its last iterate. info: host array.
 * Errors: EINVAL for a NULL pointer or K < 1; ENOMEM; ECUDA. */
fcgno_status fcgno_krylov_harvest(fcgno_op_t A, const double* b, const double* x0,
                                  const double* u_star, int K, double* r_out, double* e_out,
                                  fcgno_solve_info* info, void* stream);

/* One training step on the energy-norm loss of Eq. (11):
 * loss = mean_b ||z_b - e_b||_A / ||e_b||_A with z_b = NO(r_b, log k_b), and its gradient
 * with respect to every weight of the blob. r, e: [batch][N][N] (batch = op's batch).
 * loss: device float scalar; grad: device float blob (same layout as the weights), both
 * overwritten. prec: FCGNO_FP32 (forward/backward on CUDA cores, FP32), FCGNO_FP64, or
 * FCGNO_BF16 (Section 2.4.1's mixed precision: the Fourier layers' forward and backward run
 * on the tensor cores with BF16 operands and FP32 accumulation; the encoder, decoder, loss
 * (FP64) and every weight-gradient reduction run in FP32 on CUDA cores). FCGNO_BF16 takes the
 * model shapes and grids of the 16-bit preconditioner (else EINVAL), keeps its saved
 * activations with the operator, and re-derives the model's BF16 weight images from the FP32
 * master blob on every call (an optimiser may change the blob between calls; the
 * preconditioner then follows the new weights without fcgno_model_sync).
 * Uses the FP32 master blob given to fcgno_model_create.
 * Errors: EINVAL for a NULL pointer, batch != op's batch, another precision or
 * N < 2*modes; ENOMEM; ECUDA. */
fcgno_status fcgno_train_step(fcgno_model_t model, fcgno_op_t op, const double* r, const double* e,
                              int batch, fcgno_prec prec, float* loss, float* grad, void* stream);

/* Activation checkpointing of fcgno_train_step / fcgno_train_step_loss (a memory option, not
 * part of the method). The forward keeps every layer's input and its (small) analysis output
 * for the backward; the layers' pre-activations (batch*N*N*width values each) are kept as well
 * (mode 2, "never recompute"), or rebuilt one layer at a time during the backward from the
 * kept input (mode 1, "always": about half the activation memory, one more mixing and
 * synthesis pass per layer, bit-identical gradients; FCGNO_BF16 also repeats the layer's
 * analysis). Mode 0 (default) recomputes when the kept pre-activations would exceed 2 GiB
 * (FP32/FP64: e.g. fine-tuning on 1024 x 1024 or 2048 x 2048 grids; FCGNO_BF16 keeps them in
 * 16 bits, half the bytes). Takes effect at the next training step. Errors: EINVAL for a NULL
 * model or another mode. */
fcgno_status fcgno_model_set_train_recompute(fcgno_model_t model, int mode);

/* Training losses. FCGNO_LOSS_ENERGY is Eq. (11) in error form (the A-norm); FCGNO_LOSS_L2
 * is the paper's ablation loss in error form, mean_b ||z_b - e_b||_2 / ||e_b||_2 (defined
 * beside Eq. (11) in Section 2.4.1 and compared with it in Section 3.4). */
typedef enum {
  FCGNO_LOSS_ENERGY = 0,
  FCGNO_LOSS_L2 = 1
} fcgno_loss;

/* fcgno_train_step with a choice of loss: identical arguments, outputs and errors, plus
 * `loss_kind` (a fcgno_loss; other values: FCGNO_EINVAL). With FCGNO_LOSS_L2 no operator
 * is applied in the loss; the op still supplies log k and the grid. */
fcgno_status fcgno_train_step_loss(fcgno_model_t model, fcgno_op_t op, const double* r, const double* e,
                                   int batch, fcgno_prec prec, int loss_kind, float* loss, float* grad,
                                   void* stream);

/* fcgno_train_step_loss in FP64 with the loss and the gradient stored in FP64 (double* loss:
 * device scalar; double* grad: device array laid out like the weight blob), for gradient checks
 * below FP32 resolution. Forward and backward run on CUDA cores in FP64 from the model's FP64
 * copy of the weights (made by fcgno_model_create / fcgno_model_sync). Arguments, loss kinds
 * and errors as fcgno_train_step_loss (no precision argument). */
fcgno_status fcgno_train_step_f64(fcgno_model_t model, fcgno_op_t op, const double* r, const double* e,
                                  int batch, int loss_kind, double* loss, double* grad, void* stream);

/* Serving buckets (continuous batching of independent solves of one grid size). A bucket
 * keeps `capacity` solves resident (operator, iterate, right-hand side and Krylov state of
 * Algorithm 1) and advances all running slots together, `iters_per_step` iterations per
 * fcgno_bucket_step (replayed as one CUDA graph after the first step). Slots are admitted
 * and retired independently; each slot's truncation window follows its own iteration
 * count, so a slot's result does not depend on the other slots. Bpc NULL = identity.
 *  - create: all slots start stopped. Errors: EINVAL, ENOMEM.
 *  - admit: copy k, f, x0 (DEVICE [N][N]) into `slot`, assemble its operator, form r_0; the
 *    slot runs from its next step on. The slot must be free (stopped).
 *  - step: asynchronous on `stream`.
 *  - poll: synchronises; fills HOST arrays of `capacity` entries: status (-1 running,
 *    FCGNO_OK converged, FCGNO_EBREAKDOWN, FCGNO_ENOCONV once iters >= max_iter), iterations,
 *    relative residual.
 *  - take: copy the slot's iterate to x_out (DEVICE [N][N], may be NULL) and stop the slot,
 *    freeing it for the next admit.
 *  - Errors: EINVAL for a NULL bucket or pointer, a slot outside 0..capacity-1, and at
 *    create N < 2 (or < 2*modes), capacity < 1, m_max outside 1..8, tol < 0 or NaN,
 *    max_iter < 1 or iters_per_step < 1; poll also ETIMEOUT (see the conventions).
 *    destroy: NULL is a no-op. */
typedef struct fcgno_bucket* fcgno_bucket_t;
fcgno_status fcgno_bucket_create(int N, int capacity, fcgno_model_t Bpc, fcgno_prec prec, int m_max, double tol,
                                 int max_iter, int iters_per_step, void* stream, fcgno_bucket_t* out);
fcgno_status fcgno_bucket_admit(fcgno_bucket_t bucket, int slot, const double* k, const double* f, const double* x0,
                                void* stream);
fcgno_status fcgno_bucket_step(fcgno_bucket_t bucket, void* stream);
fcgno_status fcgno_bucket_poll(fcgno_bucket_t bucket, int32_t* status, int32_t* iters, double* relres, void* stream);
fcgno_status fcgno_bucket_take(fcgno_bucket_t bucket, int slot, double* x_out, void* stream);
fcgno_status fcgno_bucket_destroy(fcgno_bucket_t bucket);

/* Device-driven serving of a bucket (continuous batching without a host poll per step). After
 * fcgno_bucket_serve_enable, the host only appends requests (fcgno_bucket_enqueue), launches
 * steps (fcgno_bucket_step) and collects results (fcgno_bucket_results); admission and
 * retirement run on the device at the start of EVERY iteration of every step:
 *  - a slot whose solve stopped (converged, breakdown, or iters >= max_iter) has its iterate
 *    copied into its request's x_out, then its result record is published and the slot is
 *    freed (it takes a new request from the next iteration on);
 *  - every free slot takes the next queued request (first in, first out): its operator is
 *    assembled from k, f and x0 are copied in and r_0 = f - A x0 is formed; the solve runs from
 *    that same iteration on.
 * The queue and the result ring live in pinned host memory mapped into the device's address
 * space, so neither side waits for the other: enqueue and results are host-only calls (no
 * CUDA call, no synchronisation) that any number of steps in flight may overlap. A request's
 * arithmetic is that of fcgno_bucket_admit and the slot's own solve, so its result does not
 * depend on the other requests, the slot it gets or when it is admitted.
 *  - serve_enable: allocates a queue of `queue_capacity` requests and a ring of
 *    `result_capacity` results; the bucket's slots must all be free (none admitted or taken
 *    since the last take). Errors: EINVAL (NULL bucket, capacities < 1, a slot still
 *    running, called twice), ENOMEM.
 *  - enqueue: copies *req into the queue; the device reads k, f, x0 when the request is
 *    admitted and writes x_out when it stops, so these DEVICE buffers must stay valid until
 *    the request's result has been collected. FCGNO_ENOMEM when the queue is full (retry after
 *    collecting results and stepping); EINVAL for a NULL argument or a bucket not enabled.
 *  - results: moves up to `max` published results, in completion order, into the HOST array
 *    `out` and returns their number (0 when none is ready; -1 for a NULL argument or a bucket
 *    not enabled). A result is published only after its x_out has been written. A ring that
 *    the host leaves full holds retired slots back (they stay stopped) until it drains. */
typedef struct {
  const double* k;   /* [N][N] coefficient field (device) */
  const double* f;   /* [N][N] right-hand side (device) */
  const double* x0;  /* [N][N] initial guess u_0 (device) */
  double* x_out;     /* [N][N] receives the iterate when the solve stops (device) */
  uint64_t tag;      /* the caller's identifier, returned with the result */
} fcgno_serve_request;
typedef struct {
  uint64_t tag;      /* the request's tag */
  int32_t status;    /* FCGNO_OK, FCGNO_EBREAKDOWN or FCGNO_ENOCONV */
  int32_t iters;     /* iterations performed */
  double relres;     /* ||r|| / ||r_0|| of the returned iterate (recursively updated residual) */
  uint64_t seq;      /* 1-based publication number (written last) */
} fcgno_serve_result;
fcgno_status fcgno_bucket_serve_enable(fcgno_bucket_t bucket, int queue_capacity, int result_capacity);
fcgno_status fcgno_bucket_enqueue(fcgno_bucket_t bucket, const fcgno_serve_request* req);
int fcgno_bucket_results(fcgno_bucket_t bucket, fcgno_serve_result* out, int max);

/* Device bytes fcgno_solve needs for one op of this shape, for admission against an HBM
 * budget: the assembled operator (aE, aN, diagonal, log k in FP64 and log k in FP32), the
 * Krylov workspace (r, w, Jacobi scratch, 1/diag, m_max+1 slots of p_k and s_k, per-instance
 * scalars and partial sums) and the preconditioner's buffers in `prec` (16-bit activations,
 * which belong to the operator, or the CUDA-core buffers, which belong to the model and are
 * counted here too). The count is the sum of the sizes the library allocates. A serving
 * bucket holds its slots' iterates and right-hand sides on top (2 * 8 * N * N per slot).
 * Host-only; 0 for N < 2, batch < 1 or m_max < 1; an invalid desc counts no preconditioner. */
size_t fcgno_workspace_bytes(int N, int batch, int m_max, const fcgno_model_desc* desc, fcgno_prec prec);

/* 1 if the preconditioner in precision `prec` supports model shape `desc` on an N x N grid
 * (the calls taking it would not return FCGNO_EINVAL for the shape), else 0. Host-only.
 * FCGNO_FP64 / FCGNO_FP32 take any valid desc with N >= 2*modes; FCGNO_BF16 / FCGNO_FP16 also
 * need width 16 or 32, proj_width = width and N = 32, 64 or a multiple of 128. */
int fcgno_precision_supported(int N, const fcgno_model_desc* desc, fcgno_prec prec);

/* Static text for a status. */
const char* fcgno_status_str(fcgno_status s);
/* Text of the last error set on the calling thread (thread-local; valid until that
 * thread's next failing call). */
const char* fcgno_last_error(void);
/* Number of CUDA kernels this library has launched since load (all threads). */
uint64_t fcgno_launch_count(void);

/* FP64 multiply-add rate (a measurement aid, not part of the method: on GB300 the FP64 Krylov
 * kernels of Algorithm 1 are bounded by the FP64 pipe, whose rate no vendor figure gives for
 * this part). Launches `blocks` CTAs of 256 threads on `stream`; every thread runs 8
 * independent chains x <- fma(x, a, c), started at x = 1 + j/16 (j = 0..7), for `steps` steps
 * and writes the sum of the 8 final values to out[thread] (out: blocks * 256 doubles, device,
 * caller-owned). *fmas (host) receives blocks * 256 * 8 * steps, the multiply-adds the launch
 * performs. The caller times the launch with CUDA events on `stream`; asynchronous.
 * FCGNO_EINVAL before any launch when blocks is outside 1..2^20, steps outside 1..2^24 or
 * out/fmas is NULL. */
fcgno_status fcgno_fp64_fma_rate(int blocks, int steps, double a, double c, double* out, uint64_t* fmas,
                                 void* stream);

/* Failure-detection self-test (not part of the method). Every wait of the tensor-core
 * kernels on an mbarrier (bulk copies, MMAs, hand-offs between warp roles) is bounded: after
 * about 1 s the kernel raises a timeout flag that belongs to the operator, drains its own
 * copies and MMAs, frees its tensor memory and returns; fcgno_solve and fcgno_bucket_poll then
 * read and clear the flag and return FCGNO_ETIMEOUT. This call checks that path without
 * faulting or hanging the GPU: it launches one block on `stream` whose single active thread
 * waits, through the same bounded wait with a limit of `limit_seconds` (1e-6 .. 1), for a
 * barrier phase that nothing completes (no copy, MMA or other thread arrives), raises the
 * operator's flag when the wait gives up, then reads and clears the flag (synchronising
 * `stream`). Returns FCGNO_ETIMEOUT when the wait gave up (always, unless the GPU clock
 * misbehaves), FCGNO_OK otherwise; the operator stays usable either way. FCGNO_EINVAL for a
 * NULL operator or a limit outside the range; FCGNO_ENOMEM if the flag cannot be allocated. */
fcgno_status fcgno_wait_selftest(fcgno_op_t A, double limit_seconds, void* stream);

/* Launch-shape policy of the solves and serving buckets (a performance control). 0 (default):
 * a solve replays its iterations in the wide shapes while more than 80 instances are running and
 * in the narrow shapes after (the FCG step on a cluster of CTAs per instance; the 16-bit
 * analysis, mixing and synthesis in narrower grid-column chunks: shorter serial chains when few
 * instances are left); a bucket takes the narrow shapes while at most 80 of its slots can be
 * running; 1: always wide; 2: always narrow (also fcgno_precond_apply). The shapes differ only in
 * the FCG step's summation order (FP64 rounding) and in where the 16-bit preconditioner rounds
 * its partial coefficients (within its 16-bit tolerance). Applies to calls made after it, from
 * every thread. EINVAL for another mode. */
fcgno_status fcgno_set_launch_shape(int mode);

/* Kernel tracing (not part of the method): select a kernel family by name ("tc_synthesis",
 * "tc_analysis", "tc_mix", "tc_lift", "fcg_fused", "fcg_tiled", "" = off). Every later launch
 * of that family is bracketed by two CUDA events recorded on its launch stream.
 * fcgno_trace_collect waits for the recorded events and returns the summed device time
 * (ms) and the number of traced launches since the previous collect (EINVAL for a NULL
 * output). An unknown family name traces nothing. */
fcgno_status fcgno_trace_set(const char* family);
fcgno_status fcgno_trace_collect(double* total_ms, uint64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* FCGNO_H */
