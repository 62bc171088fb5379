/*
 * bioem.h — C ABI of a GB300 (sm_103a) implementation of the BioEM scoring hot path:
 * the posterior of every particle image given a structural model, integrated over
 * orientations x PSFs x in-plane displacements (Cossio, Rohr et al., "BioEM: GPU-accelerated
 * computing of Bayesian inference of electron microscopy images", arXiv:1609.06634).
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are DEVICE pointers on the context's device, owned by the caller;
 *     the library never frees them and keeps no reference to them after the call returns.
 *     Host pointers are named without the prefix.
 *   - Images are float32, row-major [n][ny][nx] (x fastest); pixel (j, k) is at
 *     x_j = (j - nx/2) * pixel_A, y_k = (k - ny/2) * pixel_A (Eq. 1's pixel positions).
 *     Only square images with nx = ny in {32, 64, 96, 128, 192} are supported in this version.
 *   - Handles (bioem_ctx, bioem_images, bioem_projset) are owned by the library and freed by
 *     the matching bioem_free_* / bioem_destroy call.
 *   - Work is enqueued asynchronously on the context's CUDA stream (the caller's stream; not
 *     owned).  Errors detectable on the host are returned immediately; errors found by kernels
 *     (a numerically degenerate image or projection) are recorded in a device status word that
 *     bioem_get_status() reads after synchronising the stream.
 *   - Return value: BIOEM_OK (0) or a negative BIOEM_ERR_* code.  Outputs are written only when
 *     the call (and, for device-detected errors, the stream) completes without error.
 *   - No C++ exception crosses this interface.
 */
#ifndef BIOEM_H
#define BIOEM_H

#ifdef __cplusplus
extern "C" {
#endif

#define BIOEM_OK 0
#define BIOEM_ERR_INVALID_ARG (-1)      /* null pointer, negative count, mismatched handles      */
#define BIOEM_ERR_UNSUPPORTED_SIZE (-2) /* image size or shift window this build does not handle */
#define BIOEM_ERR_OOM (-3)              /* device allocation failed                              */
#define BIOEM_ERR_CUDA (-4)             /* a CUDA runtime call or kernel launch failed           */
#define BIOEM_ERR_TIMEOUT (-5)          /* a bounded device wait gave up                         */
#define BIOEM_ERR_NUMERIC (-6)          /* degenerate moments (zero variance) or |rho| >= 1      */

typedef struct bioem_ctx bioem_ctx;
typedef struct bioem_images bioem_images;
typedef struct bioem_projset bioem_projset;
typedef struct bioem_batch bioem_batch;
typedef struct bioem_cnn bioem_cnn;

/* One point of the PSF grid, in physical units (the CTF and envelope after Eq. 4).
 * Converted to the paper's coefficients as a = lambda_e * defocus_A / (2 pi),
 * A = amp_contrast, b = bfactor_A2 / (8 pi^2), lambda_e the relativistic electron wavelength
 * at voltage_kV; the defocus phase is then pi lambda_e defocus k^2 and the envelope
 * exp(-B k^2 / 4) for spatial frequency k (1/A).  No spherical aberration term. */
typedef struct {
    double defocus_A;
    double amp_contrast; /* in [0, 1] */
    double bfactor_A2;   /* >= 0 */
    double voltage_kV;   /* > 0 */
} bioem_ctf;

/* Create a context on CUDA device `device`, enqueueing work on `cuda_stream` (a cudaStream_t,
 * or NULL for the legacy default stream).  Allocates the device status word and uploads the
 * transform twiddle tables.  *out is set only on success. */
int bioem_create(bioem_ctx** out, int device, void* cuda_stream);

/* Change the stream later calls enqueue on.  Handles made earlier keep the stream that was
 * current when they were made for their release (bioem_free_images / bioem_free_projset). */
int bioem_set_stream(bioem_ctx* ctx, void* cuda_stream);

/* Upper bound (bytes) on the per-pair record buffer bioem_score uses; larger parameter sets
 * are processed in waves that fit.  Default 2 GiB. */
int bioem_set_scratch_limit(bioem_ctx* ctx, unsigned long long bytes);

/* Arithmetic of the correlation step (Sec. 3.9, single versus double precision; the paper's
 * kernels are FP32).  BIOEM_PRECISION_FP32 (default): FP32 Fourier product and pruned inverse
 * FFT on the CUDA cores.  BIOEM_PRECISION_BF16X2 / BIOEM_PRECISION_FP16X2: the inverse transform
 * restricted to the displacement window written as one dense real matrix product on the tensor
 * cores, every operand split into two 16-bit floats (hi + lo; FP16 with power-of-two scaling),
 * products hi*hi + hi*lo + lo*hi accumulated in FP32; moments and log-sum-exps stay FP64.  The
 * tensor forms need (2 max_shift + 1)^2 <= 256 and build, on first use, operand copies kept with
 * the handles (freed with them): ceil(n_ps / 128) * 128 * nx * (nx + 2) * 4 bytes for a projection
 * set and ceil(n_img / IPT) * 256 * nx * (nx + 2) * 4 bytes for images, IPT = floor(256 /
 * (2 max_shift + 1)^2) images per 256-column tile (nx^2 in place of nx (nx + 2) in real space).
 * The mode applies to bioem_score, bioem_score_all, bioem_best_params and bioem_score_pairs;
 * bioem_score_noalloc, the batched and the gathered entry points always use FP32.
 * Errors: INVALID_ARG for an unknown mode. */
#define BIOEM_PRECISION_FP32 0
#define BIOEM_PRECISION_BF16X2 1
#define BIOEM_PRECISION_FP16X2 2
/* The same tensor-core product in real space (Sec. 3.3's real-space variant, one correlation per
 * displacement): K = N^2 pixels of the zero-mean, unit-norm projection against the displaced
 * zero-mean, unit-norm image, instead of the 2 N (N/2 + 1) half-spectrum terms. */
#define BIOEM_PRECISION_BF16X2_REAL 3
#define BIOEM_PRECISION_FP16X2_REAL 4
/* The FP32 form (the pruned two-stage inverse transform of the Fourier product, Sec. 3.3) with its
 * first stage, the ky transform of every column restricted to the displacement window, run as a
 * split-precision matrix product on the tensor cores: FP16 hi + lo parts of both the transform
 * matrix and the products (all four cross terms), FP32 accumulation; the products, the kx stage,
 * the likelihood and everything after it as in the FP32 form.  128 px images, max_shift <= 16
 * only (UNSUPPORTED_SIZE otherwise); no operand copies are kept. */
#define BIOEM_PRECISION_FP16X2_FFT 5
int bioem_set_precision(bioem_ctx* ctx, int mode);
int bioem_get_precision(const bioem_ctx* ctx);

/* Failure-detection test hook (no counterpart in the paper).  Arms the next tensor-core scoring
 * launch of this context (precision BF16X2 / FP16X2 / *_REAL or FP16X2_FFT) to leave K chunk
 * skip_chunk of every block unfed: in the split-precision GEMM the producer issues no copies for
 * it, in the FP16X2_FFT form no MMAs and no commit, so the barrier that chunk's consumers wait on
 * never completes.  Every barrier wait of that launch gives up after wait_ns (1 us .. 2 s) instead
 * of the default 2 s; the kernel then raises BIOEM_ERR_TIMEOUT in the device status word, leaves its
 * loops together, waits (bounded) for the copies and MMAs it did issue, frees its tensor memory and
 * returns, and the context stays usable.  The scoring call's outputs are undefined.  One launch
 * only; skip_chunk = -1 disarms.  Errors: INVALID_ARG. */
int bioem_set_wait_test(bioem_ctx* ctx, long long skip_chunk, unsigned long long wait_ns);

/* Free the context and everything it owns (not the handles made with it). */
void bioem_destroy(bioem_ctx* ctx);

/* Read and clear the device status word: synchronises the context's stream, writes 0 or a
 * BIOEM_ERR_* code to *out_status, and returns BIOEM_OK unless the synchronisation failed. */
int bioem_get_status(bioem_ctx* ctx, int* out_status);

/* Message of the last host-side error of this context (static storage, never NULL). */
const char* bioem_last_error(const bioem_ctx* ctx);
const char* bioem_status_string(int status);

/* Image preparation (Sec. 3: the per-image constants C_o, C_oo precomputed once; Sec. 3.3:
 * the observed images' Fourier transforms precomputed once, C_oo by Plancherel's theorem).
 *   d_images [n_img][ny][nx] float32, device.  pixel_A > 0.
 * Computes, per image, the float64 moments C_o = sum o, C_oo = sum o^2, A = n C_oo - C_o^2 and
 * the zero-mean, unit-norm half spectrum used by bioem_score.  *out is a library-owned handle.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, OOM, CUDA; a zero-variance image sets NUMERIC in the
 * device status word. */
int bioem_prepare_images(bioem_ctx* ctx, const float* d_images, int n_img, int nx, int ny,
                         double pixel_A, bioem_images** out);

/* Calculated images of a model for every parameter set (Fig. 1: rotate, project, PSF; Eqs. 1,
 * 4, 5).  Parameter set p = iq * nctf + ictf.
 *   d_atoms [n_atoms][4] float32 device: x, y, z (A) and weight of isotropic Gaussian atoms of
 *           standard deviation sigma_A; the projection integrates each atom over z and over each
 *           pixel exactly (erf differences), all atoms, no cutoff, mass outside the box cropped.
 *   d_quats [nq][4] float32 device: quaternions (w, x, y, z); normalised by the library; active
 *           rotation r' = R(q) r, then projection along z'.
 *   ctfs    [nctf] HOST array of PSF grid points.
 * Stores, per parameter set, the PSF-filtered projection's unit-norm half spectrum and the
 * float64 moment B = n C_cc - C_c^2.  Memory: nq * nctf * ny * (nx/2 + 1) * 8 bytes.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, OOM, CUDA; an all-zero projection sets NUMERIC. */
int bioem_project_model(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A,
                        const float* d_quats, int nq, const bioem_ctf* ctfs, int nctf,
                        int nx, int ny, double pixel_A, bioem_projset** out);

/* Posterior of every image (Eq. 9 as a Riemann sum over the grid, uniform weights):
 *   d_logP[w] = ln( (1 / (n_ps S)) sum_{p, d} L(w | p, d) ),
 * with L the likelihood of Eq. 8 integrated in closed form over the normalisation N (real line),
 * the offset mu (real line) and the noise lambda (0, inf) under flat unit priors:
 *   ln L = (3-n)/2 ln(A B - X^2) + (n-4)/2 ln B + c(n),   X(d) = n C_co(d) - C_o C_c,
 *   c(n) = -ln 2 + (1 - n/2) ln 2 pi + ln Gamma((n-3)/2) + (n-3)/2 ln(2n),
 * C_co(d) = sum_r o(r) I1((r + d) mod N) the cyclic correlation (Sec. 3.3, Eqs. 11-12) for every
 * displacement d = (dx, dy) with |dx|, |dy| <= max_shift, S = (2 max_shift + 1)^2.
 *   d_logP            [n_img] float64 device, required.
 *   d_logP_per_orient [n_img][nq] float64 device or NULL: ln of the mean over (ctf, d) of L for
 *                     each orientation (Sec. 3.8, posterior as a function of orientation).
 * Requires images and projset with the same nx, ny, pixel_A; 0 <= max_shift < nx/2 and
 * max_shift <= 4 (nx = 32), 8 (64), 12 (96), 16 (128), 24 (192) in the FP32 form, and
 * (2 max_shift + 1)^2 <= 256 (max_shift <= 7) in the split-precision forms (bioem_set_precision).
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, OOM, CUDA; NUMERIC via the status word. */
int bioem_score(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset,
                int max_shift, double* d_logP, double* d_logP_per_orient);

/* Maximising grid parameters of every image (Sec. 3.8): the (orientation, PSF, displacement)
 * with the largest ln L, and that ln L.  Ties go to the lowest (iq, ictf, dy, dx).
 * All outputs [n_img] device arrays; any may be NULL except d_best_logL. */
int bioem_best_params(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset,
                      int max_shift, int* d_best_q, int* d_best_ctf, int* d_best_dx, int* d_best_dy,
                      double* d_best_logL);

/* Both of the above from one pass over the grid (any output but d_logP may be NULL). */
int bioem_score_all(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset,
                    int max_shift, double* d_logP, double* d_logP_per_orient, int* d_best_q,
                    int* d_best_ctf, int* d_best_dx, int* d_best_dy, double* d_best_logL);

/* Per-pair values for the parameter sets [ps_begin, ps_begin + ps_count):
 *   d_pair_max [n_img][ps_count] = max_d ln L(w | p, d)
 *   d_pair_lse [n_img][ps_count] = ln sum_d L(w | p, d)   (may be NULL)
 * float64 device arrays. */
int bioem_score_pairs(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset,
                      int max_shift, int ps_begin, int ps_count, double* d_pair_max,
                      double* d_pair_lse);

/* One chunk of a chunked (resumable) scan: folds every parameter set of `projset` into running
 * per-image accumulators d_acc [n_img][2] float64 device = (M, S) with ln sum_{p,d} L = M + ln S,
 * the state of Eq. 9's sum over the parameter sets scored so far (first != 0 starts it).  A grid
 * too large for device memory is projected and scored chunk by chunk (the paper splits the images
 * instead, Sec. 4.3); the accumulators can be copied to the host between chunks (a checkpoint) and
 * loaded again to resume, and accumulators of disjoint chunks merge with the same operator
 * (M, S) + (M', S') = (m, S e^{M - m} + S' e^{M' - m}), m = max(M, M').  After the last chunk
 * bioem_acc_logP with log_norm = ln(total parameter sets x S) gives what bioem_score gives.
 * Uses the context's precision mode.  Errors as bioem_score. */
int bioem_score_accumulate(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                           double* d_acc, int first);

/* Synthetic maps (Sec. 3.8): the PSF-filtered projection I1 = F^-1[F(I0) CTF Env] (Eq. 5) of
 * the model for n pairs (d_quats[i], ctfs[i]), written to d_out [n][ny][nx] float32 device.
 * Same model arguments as bioem_project_model; ctfs is a HOST array of n entries. */
int bioem_synthetic_maps(bioem_ctx* ctx, const float* d_atoms, int n_atoms, double sigma_A,
                         const float* d_quats, const bioem_ctf* ctfs, int n, int nx, int ny,
                         double pixel_A, float* d_out);

/* Scoring that allocates no device memory.  The paper has no counterpart: this is an addition of
 * this library for callers that may not allocate at scoring time, for example a service whose
 * device memory is reserved up front by another allocator (an extra cudaMalloc could fail or
 * fragment that reservation), or a latency-sensitive loop where cudaMalloc / cudaFree would
 * stall on device synchronisation.  Prepare the images and the parameter sets beforehand.
 * Computes exactly what bioem_score computes with d_logP_per_orient = NULL, into d_logP
 * [n_img] float64 device.  Its scratch (per-image accumulators and per-pair records) is one
 * 16 MiB array that the library reserves statically on every GPU it is loaded on, until the
 * process exits; parameter sets are processed in as many passes as that array requires.
 *   Limit: round_up(32 * n_img, 256) + 12 * n_img * nctf bytes must fit in 16 MiB, else
 *          BIOEM_ERR_UNSUPPORTED_SIZE with the sizes in bioem_last_error().
 *   Every call made outside a stream capture looks up the array's device address
 *   (cudaGetSymbolAddress) with the device current, so a device reset between calls is
 *   tolerated; a call made while the context's stream is capturing reuses the address of the
 *   last such lookup.  So make the first call on a device before any stream capture (a first
 *   call made during a capture returns BIOEM_ERR_INVALID_ARG).
 *   Every call uses the same array and leaves its contents behind (each call initialises what it
 *   reads).  Calls whose work overlaps on the GPU (other streams, other host threads or
 *   contexts) race on the array and corrupt each other's results: serialise them.
 * Other errors as bioem_score. */
int bioem_score_noalloc(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset,
                        int max_shift, double* d_logP);

/* Batched scoring of several models against several image stacks of mixed sizes (the paper's
 * ensemble setting of Eq. 10 needs P_mw for every model m and image w; Sec. 4 scores large image
 * sets against a model).  A segment is one (model m, stack k) pair: stacks[k] (prepared images of
 * 64, 96, 128 or 192 px) against projsets[m * n_stacks + k] (model m projected for stack k's size,
 * pixel and grid) with |d| <= max_shift[k] (at most N/8).  bioem_batch_create builds the work list
 * of all segments, allocates the per-pair records (12 bytes per pair of every segment) and captures
 * one persistent scoring launch plus one reduction launch in a CUDA graph; bioem_batch_run replays
 * the graph on the context's stream.  Output: d_logP_matrix [n_models][sum_k n_img_k] float32,
 * ln P(image | model) as bioem_score computes it, images of stack k in columns
 * [sum_{k'<k} n_img_k', ...).  Handles must outlive the batch.  Work items use the chunk size
 * chosen by bioem_autotune for their (size, shift window), or a default.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, OOM, CUDA. */
int bioem_batch_create(bioem_ctx* ctx, int n_models, int n_stacks, const bioem_images* const* stacks,
                       const bioem_projset* const* projsets, const int* max_shift, float* d_logP_matrix,
                       bioem_batch** out);
int bioem_batch_run(bioem_batch* batch);
long long bioem_batch_evals(const bioem_batch* batch);   /* image x parameter-set pairs per run */
void bioem_batch_free(bioem_batch* batch);

/* Tile autotuner for the batched launch: times candidate chunk sizes (parameter sets per work
 * item) on a trial slice of (images, projset) and keeps the fastest for (image size, max_shift)
 * in this process; with cache_path it first reads, and afterwards rewrites, a text file of
 * "npix shift chunk" lines.  *out_chunk (may be NULL) receives the choice. */
int bioem_autotune(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                   const char* cache_path, int* out_chunk);

/* Load an autotune cache file into this process's table without tuning (no device work).  Only
 * lines "npix shift chunk" with npix in {64, 96, 128, 192}, 0 <= shift <= npix/8 and chunk a
 * positive multiple of the batched instance's pairs per batch, at most 4096, are taken; any other
 * non-blank line is skipped (bioem_autotune then tunes that case afresh and rewrites the file with
 * valid lines only).  *n_taken / *n_skipped (either may be NULL) receive the counts.
 * Errors: INVALID_ARG (NULL path, or the file cannot be opened). */
int bioem_autotune_load(const char* cache_path, int* n_taken, int* n_skipped);

/* Scoring of per-image lists of parameter sets (the paper has no counterpart: it scores every
 * image on the full grid; this serves proposals that restrict each image to a few grid cells).
 * Image w is scored against projset sets d_ps_idx[d_offsets[w] .. d_offsets[w+1]) (CSR, device
 * int arrays; at most max_per_image per image), every displacement |d| <= max_shift, and the
 * results are folded into d_acc [n_img][2] float64 device = running (max, sum exp(. - max)) of
 * ln L over everything scored so far; first != 0 overwrites d_acc instead of folding into it.
 * bioem_acc_logP turns the accumulators into ln P: d_logP[w] = max + ln sum - log_norm (pass
 * log_norm = ln(number of sets scored per image x S)).  Calling it over several projection sets
 * (waves of grid cells) accumulates one posterior. */
int bioem_score_gathered(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                         const int* d_offsets, const int* d_ps_idx, int nnz, int max_per_image, double* d_acc,
                         int first);
int bioem_acc_logP(bioem_ctx* ctx, const double* d_acc, int n_img, double log_norm, double* d_logP);

/* Merge of accumulators of disjoint parts of a grid (Eq. 9's sum split over chunks of parameter
 * sets, or over the ranks of a sharded scan): d_parts [n_parts][n][2] float64 device, each
 * (M, S) with ln sum L = M + ln S (an empty part has M = -inf, S = 0); writes the (M, S) of the
 * union to d_out [n][2] float64 device, folding the parts in index order with
 * (M, S) + (M', S') = (m, S e^{M - m} + S' e^{M' - m}), m = max(M, M') (deterministic).  d_out
 * may be d_parts (the first part is overwritten).  Errors: INVALID_ARG, CUDA. */
int bioem_acc_merge(bioem_ctx* ctx, const double* d_parts, int n_parts, int n, double* d_out);

/* Log-sum-exp of consecutive groups: d_out[g] = ln sum_{j < group_len} exp(d_values[g group_len + j])
 * for g < n_groups (float64 device arrays, max-shifted; a group of -inf gives -inf).  Serves sums
 * of Eq. 9 over a few grid points, e.g. ln sum over the B-factors of one orientation and defocus of
 * the per-pair values of bioem_score_gathered_pairs.  Errors: INVALID_ARG, CUDA. */
int bioem_group_logsumexp(bioem_ctx* ctx, const double* d_values, long long n_groups, int group_len,
                          double* d_out);

/* Per-pair values of the same per-image lists (for re-ranking candidates): d_pair_lse [nnz] float64
 * device, d_pair_lse[i] = ln sum_d L(w | d_ps_idx[i], d) for the image w whose list holds entry i.
 * Arguments and errors as bioem_score_gathered. */
int bioem_score_gathered_pairs(bioem_ctx* ctx, const bioem_images* images, const bioem_projset* projset, int max_shift,
                               const int* d_offsets, const int* d_ps_idx, int nnz, int max_per_image,
                               double* d_pair_lse);

/* Posterior of a weighted ensemble of models given a set of images (Sec. 2, Eq. 10):
 *   ln P(M | Omega) = sum_w ln sum_m w_m P_mw   (up to a constant shared by all weightings),
 * from d_logP [n_models][n_img] = ln P_mw as bioem_score or the batched matrix gives it (device;
 * float64 if elem_bytes == 8, float32 if 4).  d_weights [n_models] float64 device: weights w_m >= 0,
 * normalised to sum 1 in place (all zero or negative: NUMERIC in the status word, uniform used).
 * With n_iter > 0, n_iter expectation-maximisation steps
 *   r_mw = w_m P_mw / sum_m' w_m' P_m'w,   w_m <- (1 / n_img) sum_w r_mw
 * first replace d_weights by weights of higher ensemble posterior (the objective is concave in w;
 * the paper poses the weighting problem without an optimiser: this iteration is the textbook one
 * for weights of fixed mixture components).  Outputs, float64 device:
 *   d_out[0]      ln P(M | Omega) at the final weights;
 *   d_out[1 + m]  sum_w ln P_mw, the log posterior of model m alone (its rank among the models).
 * Sums run in a fixed order (deterministic).  1 <= n_models <= 512, n_img >= 1.
 * Errors: INVALID_ARG, OOM, CUDA. */
int bioem_ensemble(bioem_ctx* ctx, const void* d_logP, int elem_bytes, int n_models, int n_img, double* d_weights,
                   int n_iter, double* d_out);

/* Learned orientation / defocus proposal (no counterpart in the paper).  A convolutional network
 * on the image averaged over downsample x downsample pixels and standardised: six 3x3 convolutions
 * of `channels` channels (strides 1, 2, 1, 2, 1, 2; ReLU), then two linear heads: n_qbins coarse
 * orientation bins and n_dbins defocus bins.  Trained by the library's own forward / backward
 * kernels (cross-entropy of both heads, Adam on float32 master weights, float16 weights in the
 * passes).  image_px / downsample must be a multiple of 8; batches hold at most max_batch images
 * [B][image_px][image_px] float32 (device).  Flat parameter order: per conv layer W[co][ci][3][3],
 * b[co]; then Wq[n_qbins][F], bq, Wd[n_dbins][F], bd, F = channels (image_px/downsample/8)^2.
 *   bioem_cnn_create      counter-based uniform initialisation from `seed` (biases zero)
 *   bioem_cnn_gradients   loss per sample [B] and all gradients (mean over the batch) [n_params]
 *   bioem_cnn_train_step  gradients then one Adam step with learning rate lr
 *   bioem_cnn_forward     logits [B][n_qbins], [B][n_dbins] (either may be NULL)
 *   bioem_propose         for n images (any count; processed in batches), the k joint bins
 *                         q * n_dbins + d with the largest log_softmax(q) + log_softmax(d), best
 *                         first, ties to the lower bin: d_bins [n][k] int, d_scores [n][k] (may be NULL)
 * Errors: INVALID_ARG, OOM, CUDA. */
int bioem_cnn_create(bioem_ctx* ctx, int image_px, int downsample, int channels, int n_qbins, int n_dbins,
                     int max_batch, unsigned long long seed, bioem_cnn** out);
long long bioem_cnn_num_params(const bioem_cnn* cnn);
int bioem_cnn_set_params(bioem_cnn* cnn, const float* d_params);
int bioem_cnn_get_params(bioem_cnn* cnn, float* d_params);
int bioem_cnn_forward(bioem_cnn* cnn, const float* d_images, int B, float* d_logits_q, float* d_logits_d);
int bioem_cnn_gradients(bioem_cnn* cnn, const float* d_images, const int* d_label_q, const int* d_label_d, int B,
                        float* d_grads, float* d_loss);
int bioem_cnn_train_step(bioem_cnn* cnn, const float* d_images, const int* d_label_q, const int* d_label_d, int B,
                         float lr, float* d_loss);
int bioem_propose(bioem_cnn* cnn, const float* d_images, int n, int k, int* d_bins, float* d_scores);
void bioem_cnn_free(bioem_cnn* cnn);

/* CUDA-core fused multiply-add throughput of the context's GPU (a measurement hook with no
 * counterpart in the paper: the denominator of the FP32 scoring form's roofline).  kind 0: FP32
 * fmaf, 1: FP32 packed pairs (__ffma2_rn), 2: FP64 fma.  Every SM is filled with threads running
 * 16 independent chains; `reps` timed launches of ~20 ms each (after a calibration launch) on the
 * context's stream, best kept, in flop/s (2 per multiply-add) in *flops_per_s.  Changes no clock
 * or other device setting: the figure is at whatever SM clock the device runs.
 * Errors: INVALID_ARG, CUDA. */
int bioem_fma_peak(bioem_ctx* ctx, int kind, int reps, double* flops_per_s);

/* t = ln(1 - x) as every scoring kernel evaluates it for x = rho^2, the per-displacement factor of
 * the closed-form likelihood (Eq. 8 integrated over N, mu and lambda: ln L = kA + kB + (3 - n)/2 t):
 * a five-term Taylor series for x <= 1/32, the library's log1pf above.  A test hook: d_x [n] and
 * d_t [n] float32 device arrays, 0 <= x < 1 (x = 1 gives -inf and x > 1 NaN, as log1pf does;
 * negative x are outside the contract), on the context's stream.  Errors: INVALID_ARG, CUDA. */
int bioem_ln1m(bioem_ctx* ctx, const float* d_x, long long n, float* d_t);

/* Measurement hooks.  bioem_launch_count: kernels the library has launched with this context
 * since creation or the last reset.  With timing enabled, CUDA events are recorded on the
 * context's stream around every launch; bioem_kernel_time synchronises the stream and returns the
 * summed device time (ms) and the launch count of one kernel, by name: "k_prepare_images",
 * "k_project", "k_ctf_table", "k_psf_spectra", "k_psf_real", "k_score", "k_reduce_wave",
 * "k_finalize", "k_pairs_out", "k_gemm_ops", "k_score_gemm", "k_ensemble", "k_lse_merge",
 * "k_score_tc".
 * bioem_reset_kernel_stats
 * zeroes both. */
int bioem_set_kernel_timing(bioem_ctx* ctx, int enable);
int bioem_kernel_time(bioem_ctx* ctx, const char* kernel, double* total_ms, unsigned long long* launches);
int bioem_reset_kernel_stats(bioem_ctx* ctx);
unsigned long long bioem_launch_count(const bioem_ctx* ctx);

/* Handle queries (the number of images / parameter sets; -1 for NULL) and release.
 * bioem_free_images / bioem_free_projset release the handle's device memory (spectra, per-item
 * constants and any cached split-precision operands) with stream-ordered frees on the stream that
 * was current in its context when the handle was made; work that reads the handle on another
 * stream must be ordered before that stream first.  A handle may be released before or after
 * its context is destroyed, but is used only with its own context while that context lives.
 * NULL is a no-op. */
int bioem_images_count(const bioem_images* images);
int bioem_projset_count(const bioem_projset* projset);
void bioem_free_images(bioem_images* images);
void bioem_free_projset(bioem_projset* projset);

#ifdef __cplusplus
}
#endif
#endif /* BIOEM_H */
