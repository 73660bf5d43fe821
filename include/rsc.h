/*
 * rsc.h -- C ABI of librsc, GPU rotational sparse coding (rotational OMP) for
 * NVIDIA GB300 (sm_103a).
 *
 * Method: McCann, Andrearczyk, Unser, Depeursinge, "Fast Rotational Sparse
 * Coding".  Each patch x is coded by K (atom m, angle index r, weight a)
 * triples chosen greedily by orthogonal matching pursuit (Sec. II-C, the OMP
 * call of the R-K-SVD pseudocode in Fig. "code") over the augmented
 * dictionary [S_0 D, ..., S_{R-1} D] of all atoms rotated to the angles
 * 2*pi*r/R (Eq. (rot-SC)).  Patches and atoms are given in the steerable
 * circular-harmonic basis of Sec. II-D, in which a rotation is the diagonal
 * steering matrix of Eq. (Sr): harmonic k is multiplied by exp(-i k theta).
 *
 * Coefficient layout (patches and atoms alike): half spectra of real
 * signals, float32, [k][j][re,im] with harmonics k = 0..kmax and rings
 * j = 0..J-1, i.e. (kmax+1)*J*2 floats per vector, row-major, contiguous.
 * The negative harmonics are implicit (c[j,-k] = conj(c[j,k])); the Im slot
 * of k = 0 is ignored.  The inner product is the full-spectrum one,
 * <u,v> = sum_j u_j0 v_j0 + 2 sum_{k>=1} sum_j Re(conj(u_jk) v_jk).
 *
 * Conventions: every call returns an int status (RSC_OK = 0, negative on
 * error); no call throws.  Device pointers must be 16-byte aligned and
 * belong to the current CUDA device.  Calls taking a `stream` enqueue work on
 * that cudaStream_t (NULL = legacy default stream) and return after launch;
 * the caller synchronises the stream before reading outputs.  The caller owns
 * every buffer it passes; the library owns only the rsc_dict handle and the
 * device memory behind it.  There is no CPU fallback: without a usable CUDA
 * device the calls return RSC_ERR_CUDA.
 *
 * Scratch: calls that need device scratch (rsc_encode's FP16 path, the image
 * calls, the K-SVD update) take it in stream order from a memory pool per
 * device that the library creates and owns.  The pool keeps the memory it has
 * handed out between calls, so that a call does not map it again (it is not
 * the device's default pool, whose settings the library leaves alone);
 * rsc_dict_destroy gives the unused part back.  An allocation the pool
 * cannot make gives RSC_ERR_OOM.
 */
#ifndef RSC_H
#define RSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define RSC_OK 0
#define RSC_ERR_INVALID (-1)     /* bad argument (null pointer, size, alignment, norm) */
#define RSC_ERR_OOM (-2)         /* device or host allocation failed */
#define RSC_ERR_CUDA (-3)        /* a CUDA runtime call failed (message via rsc_last_cuda_error) */
#define RSC_ERR_TIMEOUT (-4)     /* a device-side bounded wait gave up (see rsc_dict_check) */
#define RSC_ERR_UNSUPPORTED (-5) /* valid but outside the sizes this build handles */

/* Arithmetic of the scoring pass (step (a)-(c) below).  Every path re-scores
 * its candidates in double-float arithmetic and solves the least-squares
 * problem in FP64, so all paths return the same selections wherever the
 * top-two margin of the exact scores exceeds their error bound. */
#define RSC_FP32 0         /* FP32 CUDA-core contraction + angle DFT */
#define RSC_F16_RESCORE 2 /* FP16 tcgen05 tensor-core scores, candidates re-scored */
/* RSC_FP32 with the exact |G| bound pruning of the angle transform: an atom
 * whose bound |G_0| + 2 sum_k |G_k| >= max_theta |score| (triangle inequality
 * over the harmonics of Eq. (Sr)) cannot reach the window of the patch's
 * running best is not transformed.  The same codes as RSC_FP32, bit for bit;
 * on GB300 it is slower than RSC_FP32 (the transform it skips is cheap next
 * to the contraction and the bound), so it is not the default. */
#define RSC_FP32_PRUNE 3

typedef struct {
  int32_t M;    /* atoms, >= 1 */
  int32_t J;    /* radial rings, >= 1 */
  int32_t kmax; /* highest angular harmonic, >= 0 */
  int32_t R;    /* rotation angles 2*pi*r/R, r = 0..R-1, >= 1 */
} rsc_dims;

typedef struct rsc_dict rsc_dict; /* opaque, device-resident, immutable */

/*
 * rsc_dict_create -- upload a dictionary D-hat (Sec. II-D, step 2 of the
 * proposed algorithm: atoms in steerable-basis coordinates) and precompute
 * its per-angle tables (the steering factors exp(-i k 2 pi r / R) of
 * Eq. (Sr), a transposed copy for the contraction, and, for the tensor-core
 * path, the steered dictionary S_r d_m in fp16, scaled by 256).
 *   coef   : device pointer, M x (kmax+1) x J x 2 floats, atoms of unit
 *            norm (|<d,d> - 1| <= 1e-4, else RSC_ERR_INVALID); read once,
 *            the caller keeps ownership.
 *   dims   : sizes; this build supports J*(kmax+1) <= 512, kmax <= 16,
 *            R <= 128 (RSC_ERR_UNSUPPORTED otherwise).
 *   stream : stream for the uploads; the call synchronises it before return.
 *   out    : receives the handle; free it with rsc_dict_destroy.
 */
int rsc_dict_create(const float *coef, rsc_dims dims, void *stream, rsc_dict **out);

/* Free a dictionary handle (NULL is accepted).  The caller must make sure no
 * rsc_encode using it is still running. */
int rsc_dict_destroy(rsc_dict *dict);

/* Sizes of a dictionary handle. */
int rsc_dict_dims(const rsc_dict *dict, rsc_dims *dims);

/*
 * rsc_encode -- rotational OMP (Sec. II-C; Eq. (rot-SC) with the steering
 * of Eq. (Sr)) of P patches, K greedy steps each.  Every step of every patch:
 *   (a) per-harmonic contraction G_k(m) = sum_j conj(d_m[j,k]) r[j,k];
 *   (b) angle transform score(m,r) = G_0 + 2 Re sum_{k>=1} e^{ik 2 pi r/R} G_k
 *       (= <S_r d_m, residual>);
 *   (c) argmax over (m, r) of |score| (ties: smallest m*R + r), certified by
 *       double-float re-scoring of every candidate within the scoring pass's
 *       error bound of the best;
 *   (e) least squares over the selected steered atoms by an incremental FP64
 *       Cholesky factor of their Gram matrix;
 *   (d) residual x - sum_i a_i S_{r_i} d_{m_i}.
 * A patch stops early (remaining outputs atom = angle_idx = -1, angle = 0,
 * coef = 0) when max |score| <= 1e-10 ||x|| or when the new pivot^2 of the
 * Cholesky factor is <= 1e-12 times its Gram diagonal entry.
 *   dict      : dictionary handle.
 *   x         : device, P x (kmax+1) x J x 2 floats.
 *   P         : patches, >= 0 (0 is a no-op).
 *   K         : greedy steps, 1 <= K <= 16.
 *   prec      : RSC_FP32, RSC_FP32_PRUNE or RSC_F16_RESCORE.  RSC_F16_RESCORE takes packed
 *               lengths J (2 kmax + 1) <= 256 and K <= 8 (RSC_ERR_UNSUPPORTED
 *               otherwise); the dictionary's tables for it are built by
 *               rsc_dict_create when the sizes allow.
 *   atom      : device int32 [P x K], atom index m per step, -1 if none.
 *   angle_idx : device int32 [P x K], angle index r in [0, R), -1 if none.
 *   angle     : device float [P x K] or NULL, the angle 2*pi*r/R in radians.
 *   coef      : device double [P x K], least-squares weights a_i (FP64).
 *   resid_norm2 : device float [P] or NULL, ||x - sum_i a_i S_{r_i} d_{m_i}||^2.
 *   stream    : cudaStream_t (NULL = default stream).
 * Outputs are in selection order.  Returns after launch.
 */
int rsc_encode(const rsc_dict *dict, const float *x, int64_t P, int32_t K, int32_t prec,
               int32_t *atom, int32_t *angle_idx, float *angle, double *coef,
               float *resid_norm2, void *stream);

/*
 * rsc_ksvd_update -- one rotational K-SVD dictionary update (the atom loop
 * of the R-K-SVD pseudocode, Fig. "code", Sec. II-C) from given codes.
 * For every atom m, each patch whose code uses m at angle r0 contributes the
 * column S_{-r0}(x_p - D_aug b_p), b_p = the patch's code without that (m, r0)
 * entry; the new atom is the first left singular vector of those columns,
 * computed as the leading eigenvector of their covariance (FP32 products,
 * FP64 sums, FP64 power iteration from the old atom, to convergence or 5000
 * iterations).  All atoms are updated from the dictionary `dict` and the same
 * codes.  Readings of the paper: a patch using m more than once contributes
 * its occurrence with the largest |weight| (ties: earliest); an atom used by
 * no patch is reset to the unit-normalised patch with the largest coding
 * error (several: successive patches in descending error; at most 64
 * resets, further unused atoms keep their old value); the largest-magnitude
 * packed entry of each new atom is positive.
 *   dict      : the dictionary the codes refer to.
 *   x         : device, P x (kmax+1) x J x 2 floats (the coded patches).
 *   P, K      : patches (>= 1) and code length (1..16).
 *   atom, angle_idx, coef : device codes as written by rsc_encode (P x K).
 *   new_coef  : device output, M x (kmax+1) x J x 2 floats, unit-norm atoms
 *               (pass it to rsc_dict_create for the next iteration).
 *   n_used    : device int32 [M] or NULL: patches that used each atom.
 *   stream    : cudaStream_t.  Returns after launch; scratch comes from the
 *               library's scratch pool (see the top of this file).
 */
int rsc_ksvd_update(const rsc_dict *dict, const float *x, int64_t P, int32_t K,
                    const int32_t *atom, const int32_t *angle_idx, const double *coef,
                    float *new_coef, int32_t *n_used, void *stream);

/*
 * rsc_ksvd_accumulate / rsc_ksvd_finish -- rsc_ksvd_update in two halves, for
 * patches spread over several GPUs (the one exchange step of the R-K-SVD
 * iteration, Fig. "code": every atom's columns come from every patch).  Each
 * rank accumulates over its own patches; the caller sums C and count over the
 * ranks (an all-reduce), merges the ranks' top lists into one list in
 * descending error (ties: smaller global patch index) and calls finish with
 * the sums on every rank; with one rank this is exactly rsc_ksvd_update.
 * rsc_ksvd_accumulate:
 *   dict, x, P, K, atom, angle_idx, coef : as rsc_ksvd_update (this rank's
 *               patches and codes).
 *   C         : device double [M][n][n] output, n = J (2 kmax + 1): the sum
 *               over this rank's columns of y y^T in the packed coordinates
 *               (overwritten).
 *   count     : device int32 [M] output: this rank's columns per atom.
 *   top_err, top_idx, top_vec : device outputs, ntop entries: this rank's
 *               patches of largest coding error ||x - D_aug b||^2 (float),
 *               descending, ties: smaller index; their local indices (int64,
 *               -1 past the end of a short list) and the patches
 *               unit-normalised (float [ntop][kmax+1][J][2]).
 *   ntop      : 0..64.
 * rsc_ksvd_finish:
 *   C, count  : device, the sums over the ranks.
 *   top_idx, top_vec, ntop : device, the merged list (top_idx only tells
 *               valid entries, >= 0, from missing ones); the i-th atom with
 *               count 0 takes the i-th valid entry, later unused atoms keep
 *               their old value.
 *   new_coef, n_used : as rsc_ksvd_update (n_used = count).
 * Both return after launch; rsc_ksvd_accumulate takes its per-patch scratch
 * from the library's scratch pool, rsc_ksvd_finish allocates nothing.
 */
int rsc_ksvd_accumulate(const rsc_dict *dict, const float *x, int64_t P, int32_t K,
                        const int32_t *atom, const int32_t *angle_idx, const double *coef,
                        double *C, int32_t *count, float *top_err, int64_t *top_idx,
                        float *top_vec, int32_t ntop, void *stream);
int rsc_ksvd_finish(const rsc_dict *dict, const double *C, const int32_t *count,
                    const int64_t *top_idx, const float *top_vec, int32_t ntop, float *new_coef,
                    int32_t *n_used, void *stream);

/*
 * Steerable basis and projection (Sec. II-D; steps 1-2 of the proposed
 * algorithm, Sec. II-E).  rsc_basis_create builds on the host, in FP64, the
 * basis of circular N x N patches (pixels with distance <= N/2 from the
 * centre): J Gaussian radial rings (centres j * ring_spacing, j = 1..J,
 * width ring_width; <= 0 selects the defaults (N-1)/(2J) and 1 pixel) times
 * the harmonics e^{i k phi}, |k| <= kmax, orthonormalised within each k, and
 * its analysis operator (pseudo-inverse of the synthesis matrix; singular
 * values up to 1e-3 of the largest are treated as zero, which bounds the
 * operator's norm by 1e3 / sigma_max), then uploads it to the current device.  Pixel (row, col)
 * of a window lies at x = col - (N-1)/2, y = (N-1)/2 - row.
 *   Limits: N <= 64, kmax <= 16, (kmax+1)*J <= 512 (RSC_ERR_UNSUPPORTED);
 *   rings that are linearly dependent on the grid give RSC_ERR_INVALID.
 */
typedef struct rsc_basis rsc_basis; /* opaque, device-resident, immutable */
int rsc_basis_create(int32_t N, int32_t J, int32_t kmax, double ring_width, double ring_spacing,
                     rsc_basis **out);
int rsc_basis_destroy(rsc_basis *basis);
/* Masked pixels per window and packed coefficient count J (2 kmax + 1). */
int rsc_basis_info(const rsc_basis *basis, int32_t *npix, int32_t *n);

/*
 * rsc_project -- coefficients x_hat = Phi^+ x of every stride-1 N x N window
 * of one image (device, h x w floats, row-major), written to `coef` (device,
 * (h-N+1)(w-N+1) x (kmax+1) x J x 2 floats, windows in row-major order of
 * their top-left corner; the layout rsc_encode takes).  Images smaller than
 * N give no windows.  Synchronises `stream` before returning.
 */
int rsc_project(const rsc_basis *basis, const float *image, int32_t h, int32_t w, float *coef,
                void *stream);

/*
 * rsc_encode_images -- rotational OMP of every stride-1 window of a list of
 * images of different sizes: one projection launch over all images (a prefix
 * sum of the window counts maps each thread to its image) into scratch
 * memory, then rsc_encode of all windows at once.
 *   images : HOST array of n_images DEVICE pointers (h[i] x w[i] floats);
 *   h, w   : HOST arrays; images smaller than the basis give no windows.
 *   basis  : must have the dictionary's J and kmax.
 *   outputs: as rsc_encode, for all windows concatenated image by image,
 *            row-major within an image.
 * Synchronises `stream` before returning.
 */
int rsc_encode_images(const rsc_dict *dict, const rsc_basis *basis, const float *const *images,
                      const int32_t *h, const int32_t *w, int32_t n_images, int32_t K,
                      int32_t prec, int32_t *atom, int32_t *angle_idx, float *angle,
                      double *coef, float *resid_norm2, void *stream);

/*
 * rsc_workspace_bytes -- device memory that one rsc_encode (basis = NULL) or
 * rsc_encode_images (basis given; P = the windows of its n_images images)
 * call takes from the library's scratch pool for its own scratch while it
 * runs, for P patches, K steps and precision prec.  The paper has no
 * counterpart: a server uses it to admit requests by the device memory they
 * need (inputs and outputs, which the caller allocates, come on top).
 *   bytes : HOST, receives the count (0 when the call needs no scratch).
 *   RSC_ERR_INVALID for null handles or pointers, P < 0, n_images < 0, K
 *   outside 1..16 or an unknown precision.  Touches no device memory.
 */
int rsc_workspace_bytes(const rsc_dict *dict, const rsc_basis *basis, int64_t P, int32_t n_images,
                        int32_t K, int32_t prec, uint64_t *bytes);

/*
 * rsc_classify_images -- the coding stage of the paper's texture classifier
 * (Sec. III-B): every stride-1 window of each image is projected once and
 * coded with each of C dictionaries (one learned per class); its label is
 * the dictionary that codes it with the least squared error (ties: the
 * smaller index), and the labels are counted per image.
 *   dicts  : C handles whose J and kmax equal the basis's (M and R may
 *            differ); 1 <= C <= 4096.
 *   images, h, w, n_images, K, prec : as rsc_encode_images.
 *   labels : device, P int32 (P = the windows of all images, image-major,
 *            row-major per image), or NULL when only the counts are wanted.
 *   hist   : device, n_images x C int32: row i counts the labels of image
 *            i's windows (zero for images smaller than a window).
 *   Device scratch: about P x ((kmax+1) J 8 + K 16 + 12) bytes from the
 *   library's scratch pool.  Synchronises `stream` before returning.
 */
int rsc_classify_images(const rsc_dict *const *dicts, int32_t C, const rsc_basis *basis,
                        const float *const *images, const int32_t *h, const int32_t *w,
                        int32_t n_images, int32_t K, int32_t prec, int32_t *labels,
                        int32_t *hist, void *stream);

/*
 * rsc_reconstruct -- the coded patches back in steerable coordinates:
 * x_hat_p = sum_i a_i S_{r_i} d_{m_i} (Sec. II-C's sparse code with the
 * steering of Eq. (Sr)), accumulated in FP64.
 *   atom, angle_idx, coef : device, P x K, as rsc_encode writes them (steps
 *            with atom = -1 are skipped); int32 / int32 / double.
 *   out    : device, P x (kmax+1) x J x 2 floats (half spectra; the Im of
 *            k = 0 is written as 0), 8-byte aligned, caller-owned.
 *   Enqueued on `stream`; returns after launch.  RSC_ERR_INVALID for bad
 *   sizes, null or misaligned pointers, or another device than the
 *   dictionary's.  For a patch x, |x - x_hat|^2 is the resid_norm2 that
 *   rsc_encode reports (up to rounding).
 */
int rsc_reconstruct(const rsc_dict *dict, int64_t P, int32_t K, const int32_t *atom,
                    const int32_t *angle_idx, const double *coef, float *out, void *stream);

/*
 * rsc_synthesize -- steerable coordinates back to pixels: pixels = Phi x_hat
 * over the basis's circular patch (step 4 of the proposed algorithm,
 * Sec. II-E: D = Phi D_hat returns a learned dictionary to the patch domain;
 * applied to rsc_reconstruct's output it gives the reconstructed patches).
 *   coef   : device, P x (kmax+1) x J x 2 floats (half spectra, the layout
 *            rsc_project writes).
 *   pixels : device, P x npix floats (rsc_basis_info's npix, the pixels with
 *            distance <= N/2 from the centre in row-major order), caller-owned.
 *   FP32 accumulation over the n packed coordinates.  Enqueued on `stream`;
 *   returns after launch.  rsc_project after rsc_synthesize gives back the
 *   coordinates' part in the span the projection keeps (the singular
 *   directions above its cutoff).
 */
int rsc_synthesize(const rsc_basis *basis, const float *coef, int64_t P, float *pixels,
                   void *stream);

/*
 * rsc_encode_host -- rsc_encode on HOST buffers (same shapes and meaning as
 * above, all pointers host memory; pinned memory gives the fastest copies).
 * Copies the patches to the device in chunks of up to 2^20, codes them and
 * copies the results back; inside a chunk each of the FP16 path's stream
 * groups copies its own patches in (one group after another) and its outputs
 * out, so that copies overlap the other groups' kernels, and with more than
 * one chunk the next chunk's work goes on a second internal stream.  Blocks
 * until every output is written.  Device staging memory (one chunk's inputs
 * and outputs, two chunks' when P > 2^20) and the two streams are made on
 * the first call and kept with the dictionary, grown when a call needs more,
 * and released by rsc_dict_destroy.  Calls on one dictionary from several
 * host threads run one at a time.
 */
int rsc_encode_host(const rsc_dict *dict, const float *x, int64_t P, int32_t K, int32_t prec,
                    int32_t *atom, int32_t *angle_idx, float *angle, double *coef,
                    float *resid_norm2);

/*
 * rsc_encode_noalloc -- the RSC_F16_RESCORE path of rsc_encode, for callers
 * that cannot allocate device memory while they code (a server that reserves
 * all of its memory up front and forbids allocation in steady state, code
 * that runs inside another framework's memory pool, or latency-bound callers
 * that must not meet an allocation failure or an allocator synchronisation
 * mid-request).  rsc_encode takes its one per-call scratch buffer (the list
 * of patches the tensor-core kernel hands to the FP32 kernel) from the
 * library's scratch pool; this call uses a fixed 4 MiB device array inside
 * the library instead and calls no cudaMalloc, cudaFree or other allocating
 * routine.  The paper has no counterpart: it is a property of this library.
 *   Arguments and outputs: as rsc_encode with prec = RSC_F16_RESCORE.
 *   Limits: P <= 1048576 (2^20) per call, else RSC_ERR_UNSUPPORTED; the
 *   dictionary must support the tensor-core path (packed length <= 112,
 *   K <= 8), else RSC_ERR_UNSUPPORTED.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress), at which point the CUDA runtime may load the
 *   array into device memory; make that first call during set-up, before
 *   any stream capture.  Later calls take no device memory.
 *   Every call on a device shares the one array and overwrites it (the call
 *   clears its counter first): calls whose work may overlap on the GPU race
 *   and give wrong results, so issue them on one stream or synchronise
 *   between them.  The array stays allocated until the process exits.
 *   The looked-up address is kept for the life of the process: a
 *   cudaDeviceReset between calls is not supported (the next call would use
 *   the address of the destroyed context).
 */
int rsc_encode_noalloc(const rsc_dict *dict, const float *x, int64_t P, int32_t K,
                       int32_t *atom, int32_t *angle_idx, float *angle, double *coef,
                       float *resid_norm2, void *stream);

/*
 * rsc_dict_check -- synchronise `stream` and report the first device-side
 * error recorded by kernels that used `dict` since the last check
 * (RSC_ERR_TIMEOUT when a bounded wait gave up), then clear it.
 */
int rsc_dict_check(const rsc_dict *dict, void *stream);

/*
 * Tuning of the FP16 path (a property of this library; the paper has no
 * counterpart).  None of these changes a result: every patch is coded the
 * same way whatever the grouping or the pipeline depth.
 *   groups               : concurrent stream groups the patches of one call
 *                          are split into (1..4; default 2);
 *   group_min            : fewest patches per group (default 65536);
 *   refine_blocks_per_sm : grid cap of the per-patch kernels per SM (1..64;
 *                          default 32);
 *   score_stages         : depth of the scoring kernel's dictionary ring, one
 *                          of the two built per layout (rows of 112 slots:
 *                          4 or 2; rows of 256 slots: 4 or 3; the first is
 *                          the default; other values give RSC_ERR_INVALID);
 *   source               : output of rsc_dict_tuning: 0 default, 1 table,
 *                          2 set by rsc_dict_set_tuning (the most specific
 *                          source of any field).
 * A field of 0 means "not set".  librsc reads a table of measured winners
 * (written by the package's autotuner) when a dictionary is created: the
 * file rsc_tuning.txt beside librsc.so, or the file named by the
 * environment variable RSC_TUNING_TABLE.  Each line reads
 * "n M R K groups group_min refine_blocks_per_sm score_stages" (n = packed
 * length J (2 kmax + 1)); '#' starts a comment.  Fields are taken in the
 * order: rsc_dict_set_tuning, the table entry of the dictionary's (n, M, R)
 * and the call's K, the default.
 */
typedef struct {
  int32_t groups, group_min, refine_blocks_per_sm, score_stages, source;
} rsc_tuning;

/* Sets (t) or clears (t = NULL) the tuning overrides of `dict`; values out
 * of range give RSC_ERR_INVALID and leave the overrides unchanged. */
int rsc_dict_set_tuning(rsc_dict *dict, const rsc_tuning *t);

/* The tuning an rsc_encode with K steps on `dict` uses (every field filled;
 * `source` as above).  HOST output. */
int rsc_dict_tuning(const rsc_dict *dict, int32_t K, rsc_tuning *out);

/* Looks up (n, M, R, K) in the table file `path` (format above): fills `out`
 * with source = 1 when an entry matches, source = 0 (fields 0) when none
 * does; RSC_ERR_INVALID when the file cannot be read.  Host only. */
int rsc_tuning_table_lookup(const char *path, int32_t n, int32_t M, int32_t R, int32_t K,
                            rsc_tuning *out);

/*
 * rsc_dict_set_limits -- diagnostic limits on `dict`, for testing the error
 * paths (a property of this library; the paper has no counterpart).
 *   pipeline_wait_ns : limit of the waits between the FP16 scoring kernel's
 *            producer, MMA and epilogue warps; a wait that runs out records
 *            RSC_ERR_TIMEOUT (reported by rsc_dict_check), stops the kernel's
 *            loops and drains what it issued (those waits keep the default 2 s).
 *            The outputs of an rsc_encode that ran into it are undefined.
 *            0 = the default, 2 s.
 *   scratch_limit : largest per-call scratch (bytes) the FP16 path may take;
 *            a call that needs more returns RSC_ERR_OOM before any device
 *            work, as if the allocator had refused.  0 = no limit.
 */
int rsc_dict_set_limits(rsc_dict *dict, uint64_t pipeline_wait_ns, uint64_t scratch_limit);

/* Diagnostic count since the last call (resets): on the FP32 path, the
 * patch-steps in which a lane discarded a candidate inside the error bound,
 * so that the step was decided by an exact re-scan of all M*R candidates; on
 * the FP16 path, the patches whose certification window held more than the
 * kept candidates and which were finished by the FP32 path. */
int rsc_dict_fallback_count(const rsc_dict *dict, int64_t *count);

/*
 * Per-phase timing (diagnostic).  While enabled (enable != 0), every
 * rsc_encode on `dict` records CUDA events around each kernel it launches, on
 * the stream that launches it.  The FP16 path normally codes two halves of the
 * patches on two streams so that their kernels overlap; with enable = 2 the
 * halves run one after the other on the call's stream, so that each launch's
 * time is the kernel's alone (enable = 1 keeps the overlap).
 * rsc_dict_timing waits for those events, returns the summed milliseconds
 * and launch counts per phase since the last call, and clears them.
 * Phases: 0 = scoring kernel of the call's path (the FP32 kernel, or the
 * tensor-core scoring kernel once per greedy step), 1 = FP32 hand-off kernel
 * of the tensor-core path, 2 = per-patch refine kernels of the tensor-core
 * path.  Meant for one stream at a time; timing adds two event records per
 * launch.
 */
int rsc_dict_set_timing(rsc_dict *dict, int enable);
int rsc_dict_timing(rsc_dict *dict, double ms[3], int64_t launches[3]);

/* Human-readable text of a status code (static storage). */
const char *rsc_status_string(int status);

/* Text of the last CUDA error seen by this thread inside librsc. */
const char *rsc_last_cuda_error(void);

/* ABI version, (major << 16) | minor. */
int rsc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RSC_H */
