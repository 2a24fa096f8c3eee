/*
 * gnp.h -- C ABI of the GB300 graph-neural-preconditioner library (libgnp.so).
 *
 * The library implements, as hand-written sm_103a CUDA kernels, the data-parallel hot
 * path of "Graph Neural Preconditioners for Iterative Solutions of Sparse Linear
 * Systems" (Chen, ICLR 2025):
 *   - the GNP operator z = M(v): scaling s (Eq. 8), MLP encoder, L Res-GCONV layers
 *     over A_hat = A / gamma (Eqs. 6-7), MLP decoder, back-scaling s^{-1};
 *   - restarted flexible GMRES with M as a nonlinear right preconditioner (Sec. 2.1,
 *     Eq. 1, Algorithm 1) in float64: SpMV, CGS2 orthogonalisation (the second pass's
 *     norm gives h_{j+1,j} = sqrt(||w1||^2 - ||h2||^2), so a step takes two grid-wide
 *     reductions), Givens QR of the Hessenberg matrix;
 *   - GNP training (Sec. 2.2, Eq. 5, Sec. 3 "Hyperparameters"): the Arnoldi/Gaussian
 *     training-pair sampler, forward, l1 residual loss, hand-written backward, Adam;
 *   - a continuous-batching solve server on top of the solver.
 *
 * Conventions shared by every call
 *   - Every call returns a gnp_status (0 = GNP_OK) and never aborts.  On failure
 *     gnp_last_error() returns a message for the calling thread.
 *   - Pointers named *_dev are device pointers owned by the caller, valid on the
 *     current CUDA device; pointers named *_host are host pointers owned by the caller.
 *     The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Work is enqueued on that stream; calls documented "synchronous" wait for it.
 *   - Objects returned through gnp_*_create are owned by the library and released by
 *     the matching gnp_*_destroy.  They allocate device memory at creation; calls that
 *     allocate later say so.
 *   - Sparse matrices are CSR with int32 row_ptr[n+1] (row_ptr[0] = 0, nondecreasing),
 *     int32 col[nnz] (0 <= col < n; any order within a row; duplicates are summed) and
 *     float64 val[nnz].
 *   - Hidden width d = 16 and MLP hidden width 32 are fixed (Sec. 3 "Hyperparameters").
 *
 * Weight blob (float32, count = gnp_weight_count(L)), every matrix row-major and applied
 * from the right (y = x W + b, with W of shape d_in x d_out as in Sec. 2.3):
 *   enc_W1[1*32], enc_b1[32], enc_W2[32*16], enc_b2[16],
 *   for l in 0..L-1: U_l[16*16], W_l[16*16],
 *   dec_W1[16*32], dec_b1[32], dec_W2[32*1], dec_b2[1].
 * The residual layer form ignores U_l but keeps its slot.
 */
#ifndef GNP_H
#define GNP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GNP_D 16
#define GNP_MLP_HIDDEN 32
#define GNP_MAX_LAYERS 32
#define GNP_MAX_RESTART 128
#define GNP_MAX_BATCH 64
#define GNP_MAX_RHS 8             /* right-hand sides of one fgmres_solve_multi call */
#define GNP_MAX_RESTART_MULTI 64  /* restart length of fgmres_solve_multi */

typedef enum {
  GNP_OK = 0,
  GNP_ERR_INVALID_ARG = 1,       /* bad argument (null pointer, size out of range) */
  GNP_ERR_INVALID_CSR = 2,       /* CSR structure violates the conventions above */
  GNP_ERR_OOM = 3,               /* device allocation failed */
  GNP_ERR_CUDA = 4,              /* a CUDA runtime call failed (message has details) */
  GNP_ERR_BREAKDOWN = 5,         /* Arnoldi breakdown with no usable direction */
  GNP_ERR_STAGNATION = 6,        /* two restart cycles without residual decrease */
  GNP_ERR_RESIDUAL_MISMATCH = 7, /* Givens residual met tol three cycles running while
                                    the true residual did not (Sec. 4 "solution failure") */
  GNP_ERR_NOT_CONVERGED = 8,     /* maxiters reached before rtol */
  GNP_ERR_TIMEOUT = 9,           /* a bounded wait or a solve's time limit expired */
  GNP_ERR_NAN = 10,              /* a NaN/Inf appeared in the iteration */
  GNP_ERR_BUSY = 11              /* server: no capacity for the request right now */
} gnp_status;

typedef enum {
  GNP_LAYER_PAPER = 0, /* Res-GCONV(X) = ReLU(X U + A_hat X W)         (Eq. 7) */
  GNP_LAYER_RESID = 1  /* X + ReLU(A_hat X W)                          (residual variant) */
} gnp_layer_form;

typedef enum {
  GNP_H_FP32 = 0, /* hidden block stored in float32 */
  GNP_H_BF16 = 1  /* hidden block stored in bfloat16 (round-to-nearest-even), float32
                     accumulation and weights */
} gnp_hprec;

typedef enum {
  GNP_PRECOND_IDENTITY = 0, /* z = v (plain GMRES) */
  GNP_PRECOND_GNP = 1,      /* z = M(v), the graph neural preconditioner (Sec. 2.3) */
  GNP_PRECOND_JACOBI = 2,   /* z = D^-1 v, D = diag(A) (Sec. 3 "Compared methods") */
  GNP_PRECOND_GMRES = 3     /* z = GMRES(A, v): inner GMRES as a preconditioner (Sec. 3) */
} gnp_precond_kind;

typedef struct gnp_config {
  int L;            /* Res-GCONV layers, 0..GNP_MAX_LAYERS (paper: 8) */
  int form;         /* gnp_layer_form */
  int hprec;        /* gnp_hprec used by gnp_apply / fgmres_solve */
  int batch;        /* training batch B: a power of two in [4, GNP_MAX_BATCH] (paper: 16) */
  int arnoldi_m;    /* Arnoldi steps of the Eq. 5 sampler, 1..64 (paper: 40) */
  float lr;         /* Adam learning rate (paper: 1e-3) */
  float beta1, beta2, eps; /* Adam constants (0.9, 0.999, 1e-8) */
  unsigned long long seed; /* Philox key of all training draws */
  /* Ablations of Sec. 4 ("Are the proposed training-data generation and the
   * scale-equivariance design necessary?"); zero = the paper's method: */
  int sample_mode;  /* 0: B/2 Eq. 5 pairs + B/2 with x ~ N(0, I);  1: x ~ N(0, I) for all B;
                       2: b ~ N(0, I) for all B (the loss then needs no x) */
  int no_scale;     /* 1: drop the scaling s of Eq. 8 (u = b, z = network output) */
} gnp_config;

typedef struct gnp_solve_info {
  int iters;            /* Arnoldi steps taken (applications of M) */
  int restarts;         /* completed restart cycles that did not converge */
  int status;           /* gnp_status of the solve (also the return value) */
  double rel_res_est;   /* last Givens residual estimate / ||b|| */
  double rel_res_true;  /* ||b - A x|| / ||b|| of the returned x */
  double seconds;       /* wall time of the solve, device-synchronised */
  /* optional outputs, owned by the caller, may be NULL: */
  double* res_history;  /* [maxiters+1]: relative residual after each iteration
                           (entry 0 = initial); res_history_len receives the count */
  int res_history_len;
  double* hessenberg;   /* [(restart+1)*restart] column-major H_bar of the last cycle */
  int hessenberg_cols;  /* receives the number of valid columns of it */
  int cycles;           /* restart cycles launched */
  int gconv_launches;   /* Res-GCONV launches timed (gnp_profile_gconv on), else 0 */
  double gconv_ms;      /* their summed CUDA-event time in milliseconds */
  double* time_history; /* optional, caller-owned [maxiters+1] (may be NULL): elapsed
                           seconds of the solve at each iteration, read from the device
                           clock (%globaltimer) by the kernel that ends the iteration;
                           entry 0 = when the initial residual was known; the t_i of the
                           Time-AUC metric (Sec. 3 "Evaluation metrics") */
} gnp_solve_info;

typedef struct gnp_mat gnp_mat;
typedef struct gnp_model gnp_model;
typedef struct gnp_server gnp_server;
typedef struct gnp_precond gnp_precond;

/* ---------------------------------------------------------------- diagnostics */

/* Human-readable name of a status code (static string). */
const char* gnp_status_string(int status);
/* Message of the last failing call on this thread (static storage, never NULL). */
const char* gnp_last_error(void);
/* Number of float32 weights for L layers: 592 + 512 L + 577. */
int gnp_weight_count(int L);

/* ---------------------------------------------------------------- matrices */

/* Copy a CSR matrix to the device.  on_device = 0: the three arrays are host
 * pointers; 1: device pointers.  The structure is validated (row_ptr monotone,
 * 0 <= col < n) before anything is allocated: violations give GNP_ERR_INVALID_CSR.
 * 1 <= n, 0 <= nnz < 2^31.  Synchronous.  The matrix also builds its transpose
 * lazily on first use by training (one extra allocation of nnz + n ints). */
int gnp_mat_create(int n, long long nnz, const int* row_ptr, const int* col,
                   const double* val, int on_device, void* stream, gnp_mat** out);
void gnp_mat_destroy(gnp_mat* A);
int gnp_mat_info(const gnp_mat* A, int* n, long long* nnz);

/* gamma = min(max_i sum_j |a_ij|, max_j sum_i |a_ij|)  (Eq. 6), computed on the
 * device in float64.  Synchronous; writes the host scalar *gamma_out. */
int gnp_gamma(const gnp_mat* A, double* gamma_out, void* stream);

/* y = A x in float64 (the SpMV of the FGMRES step, Algorithm 1).  x_dev, y_dev:
 * device float64 [n]; they must not overlap. */
int gnp_spmv(const gnp_mat* A, const double* x_dev, double* y_dev, void* stream);

/* ---------------------------------------------------------------- GNP model */

/* Build the preconditioner for A: computes gamma and A_hat = A/gamma (Eq. 6) as
 * float32 values on the device and uploads the weight blob (weights_host, float32,
 * gnp_weight_count(cfg->L) entries).  A must outlive the model.  Synchronous. */
int gnp_create(const gnp_mat* A, const gnp_config* cfg, const float* weights_host,
               gnp_model** out);
void gnp_destroy(gnp_model* M);
/* The model's gamma (Eq. 6). */
int gnp_model_gamma(const gnp_model* M, double* gamma_out);
/* Copy the weights out: after training, the best-loss snapshot (Sec. 3 keeps the
 * model of the best training step).  *count receives the blob length; host_blob may
 * be NULL to query it.  Synchronous. */
int gnp_get_weights(gnp_model* M, float* host_blob, int* count);
/* Replace the weights (and reset the Adam state and the best-loss snapshot). */
int gnp_set_weights(gnp_model* M, const float* host_blob, int count);
/* Change the hidden-block storage precision used by gnp_apply / fgmres_solve. */
int gnp_set_hprec(gnp_model* M, int hprec);

/* z = M(v) (Sec. 2.3, Fig. 1, Eqs. 6-8) for one vector: v_dev float64 [n] (read
 * only), z_dev float32 [n].  tau = ||v||_2 = 0 gives z = 0.  Asynchronous. */
int gnp_apply(gnp_model* M, const double* v_dev, float* z_dev, void* stream);
/* As gnp_apply, and also writes the hidden blocks H^0..H^L as float32
 * [(L+1) * n * 16] (node-major, 16 contiguous per node) to hidden_dev (may be NULL). */
int gnp_apply_trace(gnp_model* M, const double* v_dev, float* z_dev, float* hidden_dev,
                    void* stream);

/* One Res-GCONV layer of Eq. 7 (Sec. 2.3 item 2), layer index `layer` in [0, L):
 * H_out = ReLU(H_in U_l + A_hat H_in W_l) (GNP_LAYER_PAPER) or
 * H_in + ReLU(A_hat H_in W_l) (GNP_LAYER_RESID), with the kernel gnp_apply runs for its
 * layers before the last.  h_in_dev / h_out_dev: caller-owned device hidden blocks,
 * node-major n x 16 (16 consecutive values per node), float32 or bfloat16 as the model's
 * current hprec says; they must not overlap (GNP_ERR_INVALID_ARG when equal).  Outputs
 * are rounded to the hidden block's precision (bfloat16: round to nearest even).
 * Asynchronous on `stream`. */
int gnp_layer_apply(gnp_model* M, int layer, const void* h_in_dev, void* h_out_dev, void* stream);

/* ---------------------------------------------------------------- training */

/* Batched forward z = M(b) for B right-hand sides stored node-major (b_dev float32
 * [n*B], element (i, k) at i*B + k); z_dev float32 [n*B].  Saves the activations in
 * the model for gnp_backward_batch (one batch at a time).  FP32 hidden block. */
int gnp_forward_batch(gnp_model* M, const float* b_dev, int B, float* z_dev, void* stream);
/* Hand-written backward of the last gnp_forward_batch: given dL/dz (float32 [n*B]),
 * writes dL/dweights (float32 [gnp_weight_count(L)]) to grad_dev (overwritten). */
int gnp_backward_batch(gnp_model* M, const float* dz_dev, float* grad_dev, void* stream);
/* Training pairs of step `step` (Sec. 3: the first B/2 columns x = V_m Z S^-1 eps of
 * Eq. 5, the rest x ~ N(0, I)), written node-major to x_dev float32 [n*B] with
 * B = cfg.batch.  The first call runs the sampler's Arnoldi process and SVD.  With
 * cfg.sample_mode 1 all B columns are x ~ N(0, I); with 2 they are b ~ N(0, I). */
int gnp_sample_batch(gnp_model* M, int step, float* x_dev, void* stream);
/* One optimisation step on given solutions x (float32 [n*B] node-major): b = A_hat x,
 * z = M(b), loss = mean |A_hat z - b| (Sec. 3), backward, Adam, best-loss snapshot.
 * *loss_out (host, may be NULL) receives the loss before the update (synchronous
 * when non-NULL). */
int gnp_train_step_pairs(gnp_model* M, const float* x_dev, int B, float* loss_out,
                         void* stream);
/* One optimisation step on the model's own sampled batch (gnp_sample_batch of the
 * model's internal step counter, then gnp_train_step_pairs). */
int gnp_train_step(gnp_model* M, float* loss_out, void* stream);
/* Run `steps` training steps back to back (no per-step host sync); *best_loss_out
 * (host, may be NULL) receives the best loss seen.  Synchronous. */
int gnp_train(gnp_model* M, int steps, float* best_loss_out, void* stream);
/* As gnp_train, and losses_out (host float [steps], may be NULL) receives every step's
 * loss (before its update), for loss curves (Sec. 4, Fig. 6). */
int gnp_train_history(gnp_model* M, int steps, float* losses_out, float* best_loss_out, void* stream);

/* Free the training state (saved activations, optimiser, sampler; about
 * (2L + 10) * n * B * 64 bytes) after copying the best-loss weights to the applied
 * set.  Training again starts a fresh optimiser.  Synchronous. */
int gnp_train_release(gnp_model* M);

/* Replace the training weights from device memory (float32 [count], count =
 * gnp_weight_count(L)); also becomes the applied (best) snapshot.  Asynchronous. */
int gnp_set_weights_device(gnp_model* M, const float* w_dev, int count, void* stream);

/* Philox4x32-10 (Salmon et al., SC'11), the generator of every training draw: out[i] =
 * philox(ctr[i], key) for `count` 4 x uint32 counters (device arrays of 4*count words).
 * Exposed so that callers can check the generator bit for bit. */
int gnp_philox4x32_10(const unsigned* ctr_dev, unsigned key0, unsigned key1, int count,
                      unsigned* out_dev, void* stream);

/* ---------------------------------------------------------------- solver */

/* Solve A x = b by restarted FGMRES(restart) with right preconditioner M (NULL =
 * identity, i.e. plain GMRES), x0 = the incoming x_dev, tolerance rtol * ||b||_2,
 * at most maxiters Arnoldi steps (Algorithm 1).  Stopping rules:
 *   - an iteration is one Arnoldi step (one application of M);
 *   - within a cycle, the step whose Givens residual estimate |g_{j+1}| <= rtol ||b||
 *     ends the cycle; so does the cycle's last step (restart) or maxiters;
 *   - h_{j+1,j} <= 1e-14 ||A z_j|| (breakdown) keeps column j and ends the cycle;
 *     a rotated diagonal <= 1e-14 ||A z_j|| (z_j in the span) drops column j;
 *   - at the cycle's end x += Z y (y from the triangular system) and the true residual
 *     r = b - A x is formed: ||r|| <= rtol ||b|| returns GNP_OK; otherwise the next
 *     cycle starts from r, except that two consecutive cycles without a decrease of ||r||
 *     give GNP_ERR_STAGNATION, three consecutive cycles whose estimate met rtol while
 *     ||r|| did not give GNP_ERR_RESIDUAL_MISMATCH, a non-finite value GNP_ERR_NAN, and
 *     maxiters reached GNP_ERR_NOT_CONVERGED;
 *   - b = 0 returns x = 0 at once.
 * b_dev, x_dev: device float64 [n].  The Krylov basis V
 * ([n*(restart+1)] float64), Z ([n*restart] float32) and the reduction scratch are
 * cached in A and grown on demand (this may allocate).  Synchronous: returns when
 * the solve has ended; `info` (may be NULL) receives the statistics.
 * Returns GNP_OK on convergence, otherwise the failure status. */
int fgmres_solve(gnp_mat* A, const double* b_dev, double* x_dev, gnp_model* M,
                 int restart, double rtol, int maxiters, gnp_solve_info* info,
                 void* stream);
/* As fgmres_solve with a time limit as well (Sec. 3 "Stopping criteria": the timed
 * comparison stops by rtol or timeout).  timeout_s > 0: the first Arnoldi step that
 * ends at or after timeout_s seconds of device time (counted from the solve's first
 * kernel) ends its cycle; x is formed from the steps so far and the solve returns
 * GNP_ERR_TIMEOUT unless the true residual meets rtol.  timeout_s = 0: no limit
 * (identical to fgmres_solve).  maxiters still bounds the steps (and sizes the history
 * buffers); pass a large value to let the time limit decide.  timeout_s < 0 or
 * >= 1e9 is GNP_ERR_INVALID_ARG. */
int fgmres_solve_timeout(gnp_mat* A, const double* b_dev, double* x_dev, gnp_model* M,
                         int restart, double rtol, int maxiters, double timeout_s,
                         gnp_solve_info* info, void* stream);

/* Solve k systems A x_r = b_r (1 <= k <= GNP_MAX_RHS) with one matrix and one
 * preconditioner M (NULL = identity; a GNP with L >= 1 and float32 hidden blocks) by
 * restarted FGMRES(restart <= GNP_MAX_RESTART_MULTI), advancing all systems in lockstep so
 * that every sparse gather (the GNP layers, the SpMV, the residual) serves all of them
 * (Sec. 4: one preconditioner for any number of right-hand sides).  B_dev and X_dev are
 * float64 [n*k] node-major: element (i, r) at i*k + r; X holds x0 on entry.  Each system
 * follows the stopping rules of fgmres_solve; one whose cycle ends early waits, inactive,
 * for the others, so its iterates and iteration count are those of a solve on its own.
 * infos (may be NULL) is an array of k gnp_solve_info (per-system optional histories as in
 * fgmres_solve; hessenberg is not filled, seconds is the shared wall time).  Synchronous;
 * returns GNP_OK when every system converged, else the first failing system's status.
 * The workspace ((restart+1) n K float64 + restart n K float32 + 32 n K float32, K = k
 * rounded up to 2, 4 or 8) is cached in A. */
/* z_r = M(v_r) for k vectors at once (the GNP kernels of fgmres_solve_multi): v_dev
 * float64 [n*k] and z_dev float32 [n*k], node-major (element (i, r) at i*k + r).  Uses the
 * multi-system workspace cached in the model's matrix.  Asynchronous. */
int gnp_apply_multi(gnp_model* M, const double* v_dev, int k, float* z_dev, void* stream);
int fgmres_solve_multi(gnp_mat* A, const double* B_dev, double* X_dev, int k, gnp_model* M,
                       int restart, double rtol, int maxiters, gnp_solve_info* infos,
                       void* stream);

/* A right preconditioner for fgmres_solve_precond (the GNP and the simple baselines
 * the paper compares it with, Sec. 3 "Compared methods"):
 *   GNP_PRECOND_IDENTITY  M and the inner arguments are ignored;
 *   GNP_PRECOND_GNP       M (not owned, must outlive P, built on A) is applied;
 *   GNP_PRECOND_JACOBI    z = v / a_ii; a row with a_ii = 0 (or no stored diagonal) uses
 *                         1 (that row passes v_i through);
 *   GNP_PRECOND_GMRES     z = one cycle of at most inner_iters (1..GNP_MAX_RESTART) GMRES
 *                         steps on A z = v from z0 = 0 (float64, CGS2, Givens), ended
 *                         early when the Givens residual estimate reaches
 *                         inner_rtol * ||v|| (paper: 10 steps, 1e-6).  Owns its own
 *                         Krylov workspace ((inner_iters + 1) * n float64 and more).
 * The library owns *out (gnp_precond_destroy).  P is bound to A. */
int gnp_precond_create(gnp_mat* A, int kind, gnp_model* M, int inner_iters, double inner_rtol,
                       gnp_precond** out);
void gnp_precond_destroy(gnp_precond* P);
/* z = P(v) for one vector: v_dev, z_dev float64 [n] device arrays (distinct).
 * Asynchronous on `stream`. */
int gnp_precond_apply(gnp_precond* P, const double* v_dev, double* z_dev, void* stream);
/* fgmres_solve_timeout with any preconditioner P (NULL = identity).  With the GNP the
 * directions Z are float32 (the network's output precision); with Jacobi and inner
 * GMRES they are float64. */
int fgmres_solve_precond(gnp_mat* A, const double* b_dev, double* x_dev, gnp_precond* P,
                         int restart, double rtol, int maxiters, double timeout_s,
                         gnp_solve_info* info, void* stream);

/* The paper's convergence metrics (Sec. 3 "Evaluation metrics"), computed on the host
 * from a solve's histories (len = res_history_len = iters + 1 entries):
 *   Iter-AUC = sum_{i=0}^{iters} (log10 r_i - log10 rtol),
 *   Time-AUC = sum_{i=1}^{iters} (log10 r_i - log10 rtol) (t_i - t_{i-1}).
 * r_i <= 0 counts as the smallest normal double (2.2e-308).  len < 1, rtol <= 0 or a
 * NULL array gives NaN.  Pure host functions: no device work. */
double gnp_iter_auc(const double* res_history, int len, double rtol);
double gnp_time_auc(const double* res_history, const double* time_history, int len, double rtol);

/* ---------------------------------------------------------------- solve server */

/* Continuous batching of many FGMRES solves on one GPU (Sec. 4: one preconditioner
 * serves any number of right-hand sides; here also many matrices at once).  A server
 * thread admits queued requests in FIFO order while fewer than max_active run and their
 * device-memory footprint (Krylov basis n*(restart+1) float64, directions n*restart
 * float32, GNP hidden blocks 2*n*16 float32, reduction scratch) fits in max_bytes.
 *
 * Per-request mode (grouped = 0): every running request has its own stream and its
 * restart cycle captured as a CUDA graph; whenever one of its cycles ends, the server
 * applies its stopping rules and launches its next cycle or retires it at once, without
 * waiting for the other requests.  Results are the same as a lone fgmres_solve of the
 * request.
 *
 * Grouped mode (grouped = 1): requests whose GNP runs on the short-row layer kernels (every
 * row of A at most 16 nonzeros, L >= 1), at most 16 at once, advance together one FGMRES
 * step per round on one stream: each kernel of the step (encoder, Res-GCONV layers, SpMV
 * with CGS2 pass 1, pass 2, and the cycle end: x update and residual for the requests
 * whose restart cycle ends in that round) is launched once for all of them over a work
 * table of the requests' own grids.  The stopping rules run on the device at each cycle
 * end, so eight rounds are captured as one CUDA graph per set of running requests and
 * requests are admitted and released between launches of it (every eight steps).  Each
 * grouped request computes exactly what a lone fgmres_solve computes with the two-pass
 * CGS2 schedule (GNP_ORTHO=cgs2 in the environment); the other requests run as in
 * per-request mode. */
typedef struct gnp_server_config {
  size_t max_bytes; /* device-memory budget for the running requests' workspaces */
  int max_active;   /* requests running at once (slots) */
  int restart;      /* FGMRES restart length of every request */
  int grouped;      /* 1: grouped steps for the requests that allow them; 0: per request */
} gnp_server_config;

typedef struct gnp_server_stats_t {
  int queued, active;
  size_t used_bytes;
  long long rounds; /* restart cycles run (a grouped request's counted when it ends) */
  long long completed, max_active_seen;
} gnp_server_stats_t;

int gnp_server_create(const gnp_server_config* cfg, gnp_server** out);
/* Queue a solve of A x = b (x_dev holds x0) preconditioned by M (NULL = identity);
 * the buffers must stay valid until the ticket is collected.  A and M are read only
 * while the request runs (do not train M then); one model may serve many requests at
 * once.  Never blocks; *ticket identifies the request. */
int gnp_server_submit(gnp_server* S, gnp_mat* A, gnp_model* M, const double* b_dev,
                      double* x_dev, double rtol, int maxiters, long long* ticket);
/* GNP_ERR_BUSY while the request is queued or running; otherwise collects it and
 * returns its solve status (GNP_ERR_OOM if its footprint exceeds max_bytes).  info (may
 * be NULL) receives iterations, residuals and `seconds` = submit-to-finish latency. */
int gnp_server_poll(gnp_server* S, long long ticket, gnp_solve_info* info);
/* Block until the request finishes (then as poll) or timeout_s passes
 * (GNP_ERR_TIMEOUT; the request keeps running). */
int gnp_server_wait(gnp_server* S, long long ticket, double timeout_s, gnp_solve_info* info);
int gnp_server_stats(gnp_server* S, gnp_server_stats_t* out);
/* Finish the running requests, abandon the queued ones, join the server thread. */
void gnp_server_destroy(gnp_server* S);

/* ---------------------------------------------------------------- allocation-free gamma */

/* min(max row abs-sum, max column abs-sum) of a CSR matrix the caller already holds on
 * the device (row_ptr_dev int32 [n+1], col_dev int32 [nnz], val_dev float64 [nnz], the
 * conventions of gnp_mat_create), written to the device scalar *gamma_dev.  The CSR is
 * checked on the device only: every access stays inside [0, nnz) and [0, n), and
 * *gamma_dev is NaN when row_ptr does not start at 0, decreases or does not end at nnz,
 * or when a column index lies outside [0, n).  The column sums are added with float64
 * atomics, so the last bits of the result may differ from call to call (gnp_gamma sums
 * in a fixed order).  The paper has no counterpart of this call.  It serves callers
 * that must not allocate device memory when they call in: applications whose device
 * memory belongs to their own pool or arena, plug-ins that receive only a stream and
 * their host's buffers, loops that cannot take the implicit synchronisation of
 * cudaMalloc/cudaFree.  It allocates nothing: its scratch (column sums, block partials,
 * a counter, an error flag) is one fixed array of 8,398,592 bytes (8 MiB + 9,984 B)
 * inside the library, held by every GPU that loads the library until the process exits,
 * so n <= 1,048,576 (larger n gives GNP_ERR_INVALID_ARG).  The first call on each device
 * looks up that array's device address (cudaGetSymbolAddress) and caches it for the life
 * of the process; make that first call before any stream capture, and do not reuse the
 * library on a device after cudaDeviceReset.  Every call clears the scratch it uses and
 * shares the one array: calls that overlap on the GPU (other streams, other threads)
 * race.  Asynchronous on `stream`. */
int gnp_gamma_noalloc(int n, long long nnz, const int* row_ptr_dev, const int* col_dev,
                      const double* val_dev, double* gamma_dev, void* stream);

/* Time every Res-GCONV launch of the following solves with CUDA events recorded on
 * the solve's stream around the launch (inside the captured restart cycle); the sums
 * arrive in gnp_solve_info.gconv_ms / gconv_launches.  The event records add a little
 * time to the solve, so keep it off when timing the solve itself.  Process-wide. */
int gnp_profile_gconv(int on);

/* How many bounded device-side waits have given up since the last reset (reset != 0
 * clears the count after reading it), or -1 when the count cannot be read.  The
 * TMA-gather Res-GCONV layer (Sec. 2.3, Eq. 7; used on matrices with rows of more than 16
 * nonzeros when GNP_GCONV_TMA=1 is set) waits for its copies on mbarriers with a limit of
 * 2 s of device time; a block that reaches the limit counts it here, waits (again
 * bounded) for its copies still in flight and returns, leaving its output rows
 * unwritten.  A non-zero count means the results of the launches since the last reset
 * are not to be used.  Synchronous (reads a device counter). */
int gnp_kernel_faults(int reset);

#ifdef __cplusplus
}
#endif

#endif /* GNP_H */
