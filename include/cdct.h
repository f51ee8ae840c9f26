/*
 * cdct.h -- C ABI of the GB300 library for the blockwise 2-D DCT
 * approximations of arXiv 2207.11638 ("DCT Approximations Based on Chen's
 * Factorization").
 *
 * The library applies, to every N x N block of a batch of images, the
 * JPEG-like pipeline of Sec. 5.1:
 *
 *     forward   B  = C A C^{-1}            (C = S T, Sec. 3.1 / Sec. 6.1)
 *     zonal     keep the first r coefficients of B in zig-zag order
 *     inverse   A' = C^{-1} B C
 *     error     PSNR of A' against A
 *
 * with T one of the multiplierless matrices
 *     T~_N  (CDCT_TILDE, sign approximation, Eq. 4 and Eq. app_N),
 *     T^_N  (CDCT_HAT,   round approximation, Eq. 5 and Eq. app_N),
 * for N = 8, 16, 32 (16 and 32 by the JAM recursion of Sec. 6.1), or the
 * exact 8-point DCT-II (CDCT_EXACT, Chen's factorization Eq. 3).
 *
 * Integer variants never form B: they compute the integer coefficients
 * Y = T A U with U = N T^{-1} (an integer matrix), keep the zonal mask on Y
 * (the diagonal scale S cancels exactly in A'), and reconstruct
 * A' = (U Ym T) / N^2.  All integer stages are int32 adds and shifts; the
 * float reconstruction is the correctly rounded value of that rational.
 * With flag CDCT_CONV_TRANSPOSE the usual B = C A C^T, A' = C^{-1} B C^{-T}
 * is used instead (Y = T A T^T, A' = U Ym U^T / N^2).
 *
 * Conventions for every entry point:
 *  - Pointers to pixels, coefficients, reconstructions, PSNR outputs and
 *    workspaces are DEVICE pointers on the current CUDA device; the caller
 *    allocates and owns them.  A plan owns only host-side tables.
 *  - Calls are asynchronous and ordered on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  No entry point synchronises.
 *  - Images: rows of `width` pixels `pitch` elements apart; `batch` images
 *    `batch_stride` elements apart.  Sizes not divisible by N are padded by
 *    replicating the last row / column; outputs and the error cover the
 *    original width x height only.  CDCT_I16 pixels must lie in [-255, 255]
 *    (residuals of 8-bit frames): that range bounds every int32 intermediate.
 *  - Coefficient buffers are block-major: [batch][by][bx][N][N] (row i,
 *    column j of each block), int32 for CDCT_TILDE / CDCT_HAT, float for
 *    CDCT_EXACT.  Kept coefficients are [batch][by][bx][r] in zig-zag order.
 *  - Errors: every call returns a cdct_status.  Invalid arguments return
 *    CDCT_EINVAL before anything is launched; cdct_last_error() then gives a
 *    message (per calling thread).  CDCT_ECUDA reports a failed launch.
 */
#ifndef CDCT_H
#define CDCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cdct_plan_s* cdct_plan;

typedef enum {
  CDCT_OK = 0,
  CDCT_EINVAL = 1,        /* invalid argument; nothing launched */
  CDCT_ENOMEM = 2,        /* host allocation failed */
  CDCT_ECUDA = 3,         /* a CUDA launch or call failed */
  CDCT_EUNSUPPORTED = 4,  /* valid but not provided (e.g. EXACT with N != 8) */
  CDCT_ETIMEOUT = 5       /* a bounded device wait gave up (reported by cdct_check_device) */
} cdct_status;

typedef enum {
  CDCT_EXACT = 0,  /* exact DCT-II, N = 8 only, float32 via Eq. 3 */
  CDCT_TILDE = 1,  /* T~_N: sign() of the Chen constants (Eq. 4, Eq. app_N) */
  CDCT_HAT = 2     /* T^_N: round() of the Chen constants (Eq. 5, Eq. app_N) */
} cdct_variant;

typedef enum { CDCT_U8 = 0, CDCT_I16 = 1 } cdct_dtype;

/* plan flags */
#define CDCT_CONV_PAPER 0u      /* B = C A C^{-1}, A' = C^{-1} B C (Sec. 5.1) */
#define CDCT_CONV_TRANSPOSE 1u  /* B = C A C^T,  A' = C^{-1} B C^{-T} */

/* which matrix cdct_matrix() returns */
#define CDCT_MATRIX_T 0       /* T_N (N x N, row-major); 2 C_8 for EXACT */
#define CDCT_MATRIX_U 1       /* U_N = N T_N^{-1} (N x N); 4 C_8^T for EXACT */
#define CDCT_MATRIX_S 2       /* diag(S_N) = diag(T T^T)^{-1/2} (N values) */
#define CDCT_MATRIX_ZIGZAG 3  /* zig-zag position of (i, j) (N x N) */

/* A batch of images in device memory. */
typedef struct {
  const void* data;       /* first pixel of image 0 (device) */
  int32_t dtype;          /* cdct_dtype */
  int32_t width, height;  /* >= 1 */
  int64_t pitch;          /* elements between rows, >= width */
  int32_t batch;          /* number of images, >= 1 */
  int64_t batch_stride;   /* elements between images, >= pitch * height (ignored if batch == 1) */
} cdct_image;

/* Create a plan for block size n (8, 16, 32) and a variant; flags is
 * CDCT_CONV_PAPER or CDCT_CONV_TRANSPOSE.  *out receives the plan, which
 * the caller releases with cdct_plan_destroy.  A plan's only mutable state
 * is its pipeline schedule (cdct_plan_set_tuning); threads may share a plan
 * as long as none changes its schedule while another uses it. */
cdct_status cdct_plan_create(int n, int variant, uint32_t flags, cdct_plan* out);
cdct_status cdct_plan_destroy(cdct_plan plan);

/* Number of N x N blocks of `in` after padding (batch * nby * nbx). */
cdct_status cdct_block_count(cdct_plan plan, const cdct_image* in, int64_t* n_blocks);

/* Bytes of device workspace the PSNR-producing calls need for `in`. */
cdct_status cdct_workspace_size(cdct_plan plan, const cdct_image* in, size_t* bytes);

/* Forward transform (Sec. 5.1): coeff = Y = T A U per block (int32; float B
 * for EXACT), block-major, cdct_block_count() * N * N elements. */
cdct_status cdct_forward(cdct_plan plan, const cdct_image* in, void* coeff, void* stream);

/* Zonal retention (Sec. 5.1): in place, zero every coefficient whose
 * zig-zag position is >= r (1 <= r <= N*N).  Optional outputs (NULL to skip):
 * `scaled` = B (float, same layout): diag(s) Y diag(s)^{-1} / N (paper
 * convention) or diag(s) Y diag(s) (transpose), s = diag(S_N) of Sec. 3.1;
 * `kept` = the first r coefficients of each block in zig-zag order. */
cdct_status cdct_zonal(cdct_plan plan, int r, void* coeff, int64_t n_blocks, float* scaled,
                       void* kept, void* stream);

/* Inverse transform (Sec. 5.1): recon = (U Ym T) / N^2 for the original
 * width x height of each image; recon rows recon_pitch floats apart, images
 * recon_batch_stride floats apart. */
cdct_status cdct_inverse(cdct_plan plan, const void* coeff, int32_t width, int32_t height,
                         int32_t batch, float* recon, int64_t recon_pitch,
                         int64_t recon_batch_stride, void* stream);

/* PSNR (Sec. 5.1): psnr_db[b] = 10 log10(255^2 / MSE_b) over the original
 * pixels of image b (+inf when MSE_b = 0).  psnr_db is a device array of
 * `ref->batch` doubles; workspace needs cdct_workspace_size() bytes.  The
 * reduction order is fixed, so results are reproducible bit for bit. */
cdct_status cdct_psnr(const cdct_image* ref, const float* recon, int64_t recon_pitch,
                      int64_t recon_batch_stride, double* psnr_db, void* workspace,
                      size_t workspace_bytes, void* stream);

/* SSIM (Sec. 5.1 reports it beside PSNR; the paper cites the index of Wang
 * et al. without restating it): ssim[b] = mean over every 11 x 11 window
 * inside image b of
 *   (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
 * the statistics weighted by a unit-sum circular Gaussian window (sigma 1.5),
 * C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2, x the reference, y the
 * reconstruction.  Images must be at least 11 x 11.  ssim is a device array
 * of `ref->batch` doubles; the workspace needs cdct_ssim_workspace_size()
 * bytes (8-byte aligned).  Computed in float64 with a fixed reduction
 * order: reproducible bit for bit. */
cdct_status cdct_ssim_workspace_size(const cdct_image* ref, size_t* bytes);
cdct_status cdct_ssim(const cdct_image* ref, const float* recon, int64_t recon_pitch, int64_t recon_batch_stride,
                      double* ssim, void* workspace, size_t workspace_bytes, void* stream);

/* Fused forward -> zonal(r) -> inverse -> PSNR in one pass over the pixels.
 * recon as for cdct_inverse; kept (NULL to skip) as for cdct_zonal; psnr_db
 * (NULL to skip) as for cdct_psnr, which then needs the workspace. */
cdct_status cdct_fwd_zonal_inv(cdct_plan plan, const cdct_image* in, int r, float* recon,
                               int64_t recon_pitch, int64_t recon_batch_stride, void* kept,
                               double* psnr_db, void* workspace, size_t workspace_bytes,
                               void* stream);

/* Pipeline tuning of a plan (the autotuner sets it): staging depth of the
 * fused kernel's input ring (0 = default for N, or 1, 2, 3; N = 8 runs 1 as
 * 2; N = 16 and 32 at depth 1 are built for four resident CTAs per SM) and
 * resident CTAs per SM used for its persistent grid (0 = as many as fit).  Changes the
 * schedule only, never the results.  Not to be called while another thread
 * uses the plan. */
cdct_status cdct_plan_set_tuning(cdct_plan plan, int stages, int ctas_per_sm);

/* ---- Batches of images of uneven sizes (one persistent launch) ----------
 * A batch lists images of any sizes (device pointers; rows, widths and
 * pointers 16-byte aligned).  cdct_batch_create validates the list on the
 * host (an invalid descriptor returns CDCT_EINVAL naming the image) and
 * builds a descriptor table: the images, the prefix sums of their work units
 * and one 64-byte record per work unit (its image's pointers and geometry,
 * block row and segment, so that the kernel decodes a unit from one bulk
 * copy).  A work unit is up to
 * 128 / P blocks of one block row (P = 1, 4, 16 threads per block for N = 8,
 * 16, 32), or several whole block rows of an image at most half that wide.
 * The caller allocates `table_bytes` of device memory for it and
 * uploads it once with cdct_batch_upload; cdct_batch_fzi then runs the fused
 * forward -> zonal(r) -> inverse (+ PSNR per image) over every image in one
 * persistent launch (plus one launch for the PSNRs), which can be captured
 * in a CUDA graph.  The batch keeps the plan's N, variant and convention;
 * the plan must outlive it. */
typedef struct cdct_batch_s* cdct_batch;

typedef struct {
  const void* data;        /* first pixel (device) */
  float* recon;            /* first reconstructed pixel (device) */
  int32_t width, height;
  int64_t pitch;           /* elements between input rows */
  int64_t recon_pitch;     /* floats between reconstruction rows */
} cdct_batch_image;

cdct_status cdct_batch_create(cdct_plan plan, const cdct_batch_image* images, int n_images, int dtype,
                              cdct_batch* out);
cdct_status cdct_batch_destroy(cdct_batch batch);
/* Device bytes of the table and of the PSNR workspace; total pixels. */
cdct_status cdct_batch_sizes(cdct_batch batch, size_t* table_bytes, size_t* workspace_bytes,
                             int64_t* total_pixels);
/* Copy the table to device_table (16-byte aligned, table_bytes); synchronises `stream`. */
cdct_status cdct_batch_upload(cdct_batch batch, void* device_table, void* stream);
/* Host copy of work unit `unit`'s record (0 <= unit < the batch's work units):
 * out = {image index, first block row, segment of that row (units of up to
 * 128 / P blocks), block rows covered}.  Reads host memory only.
 * CDCT_EINVAL for a null argument or a unit out of range. */
cdct_status cdct_batch_unit(cdct_batch batch, int64_t unit, int32_t out[4]);
/* psnr_db: device array of n_images doubles (NULL to skip, then no workspace is needed). */
cdct_status cdct_batch_fzi(cdct_batch batch, const void* device_table, int r, double* psnr_db,
                           void* workspace, size_t workspace_bytes, void* stream);

/* The fused call of cdct_fwd_zonal_inv for callers that cannot allocate
 * device memory: code that must run with the buffers it already owns (a
 * fixed memory budget, no device allocator of its own, or a host that may
 * not call cudaMalloc while it runs).  It takes no workspace; the error
 * partials go to a scratch array of fixed size (1 MiB) that the library
 * holds in static device memory, on every GPU that loads it, until the
 * process exits.  The paper has no counterpart: this is an interface
 * choice, not part of the method.
 *  - Limit: with psnr_db set, a call needing more than 1 MiB of partials
 *    (cdct_workspace_size() > 1 MiB, e.g. more than about a hundred
 *    1920x1080 planes in one call) is rejected with CDCT_EINVAL; without
 *    psnr_db no scratch is used.
 *  - Set-up: the first call on a device (with that device current) looks up
 *    the scratch's device address; make that first call before any stream
 *    capture.
 *  - The scratch is shared by every call on the device: calls that overlap
 *    on the GPU (other streams, other threads) race on it and must be
 *    ordered by the caller.  Nothing in it has to start at zero: every
 *    partial a call reads is written by the same call, unless a bounded wait
 *    gives up (cdct_check_device then returns CDCT_ETIMEOUT), in which case
 *    the unfinished units' partials are written as NaN and psnr_db is NaN.
 *  - The looked-up address stays valid for the life of the device's primary
 *    context: no cdct call may follow a cudaDeviceReset of that device in
 *    the same process.
 *  - No device memory is allocated or freed by this call. */
cdct_status cdct_fwd_zonal_inv_noalloc(cdct_plan plan, const cdct_image* in, int r, float* recon,
                                       int64_t recon_pitch, int64_t recon_batch_stride, void* kept,
                                       double* psnr_db, void* stream);

/* ---- Exhaustive rate-distortion quadtree search (32 x 32 regions) -------
 *
 * The paper evaluates its 8-, 16- and 32-point transforms in a codec that
 * picks the transform size per region (Sec. 6.2) but prints no search; this
 * is the library's.  Every 32 x 32 region of the images (regions are tiled
 * from the top-left corner; pixels beyond width x height are edge-replicated
 * and excluded from the distortion) is evaluated, for each quantiser step q,
 * with all 17 quadtrees: the whole region as one 32 x 32 block, or four
 * 16 x 16 quadrants each kept or split into four 8 x 8 blocks.  Per block
 * (paper convention of Sec. 5.1, T = T~_N or T^_N, U = N T^-1):
 *   Y  = T A U; the scaled coefficients B = diag(s) Y diag(s)^-1 / N
 *        (s_i = d_i^-1/2, d = diag(T T^T), Sec. 3.1) are quantised as
 *        L = round(B / q) with the paper's round() (Sec. 3), decided exactly
 *        in integers;
 *   the decoder forms Y' = N q L c with c_ij = round(2^12 sqrt(d_i / d_j))
 *        and Z' = U Y' T (the reconstruction times 2^12 N^2);
 *   D  = sum over valid pixels of (2^12 N^2 A - Z')^2;
 *   R  = 1 (coded-block flag) + 1 per zig-zag position up to the last
 *        nonzero level + (2 floor(log2 |L|) + 2) per nonzero level;
 *   J' = (32 / N)^4 D + lambda' R with lambda' = kappa q^2 2^44 and
 *        kappa = kappa_num / 2^kappa_log2_den, i.e. J = SSE + kappa q^2 R
 *        scaled by 2^24 32^4.
 * A partition's cost adds one split-flag bit (lambda') per node that may
 * split: the region, and each quadrant when the region is split.  The label
 * minimises it; ties keep the larger transform.  Every quantity is an exact
 * integer (128-bit costs), so labels are reproducible bit for bit.
 *
 * Labels: 0 = the whole region; 1 + m = split, where bit k of m (quadrant k
 * in raster order: top-left, top-right, bottom-left, bottom-right) is set
 * when that quadrant is split into 8 x 8 blocks. */
typedef struct cdct_rd_s* cdct_rd;

/* Host tables of a variant (CDCT_TILDE or CDCT_HAT): d and c for the three
 * sizes.  Owns host memory only. */
cdct_status cdct_rd_create(int variant, cdct_rd* out);
cdct_status cdct_rd_destroy(cdct_rd rd);

/* Host copy of the tables (for tests): 1440 int32 = d_i for N = 32, 16, 8
 * (3 x 32, zero-padded), then c_ij row-major for N = 32, 16, 8. */
cdct_status cdct_rd_tables(cdct_rd rd, int32_t* out);

/* batch * ceil(width / 32) * ceil(height / 32); regions are numbered image
 * by image, row-major within an image. */
cdct_status cdct_rd_region_count(const cdct_image* in, int64_t* n_regions);

/* One launch over every region for n_q (1..4) steps q (host array, each
 * 1..4096).  kappa_num in 0..1024, kappa_log2_den in 0..44.
 *   labels          device [n_q][n_regions] uint8
 *   partition_cost  device [n_q][n_regions][17][2] uint64 (low, high words of
 *                   each partition's 128-bit J', label order), or NULL.
 * Pixels as for every entry point (CDCT_U8, or CDCT_I16 in [-255, 255]). */
cdct_status cdct_rd_search(cdct_rd rd, const cdct_image* in, const int32_t* q, int32_t n_q,
                           int32_t kappa_num, int32_t kappa_log2_den, uint8_t* labels,
                           uint64_t* partition_cost, void* stream);

/* cdct_rd_search restricted to the regions listed in region_index (device
 * int64, numbers as for cdct_rd_search); their count is read on the device
 * from *count (device int64, e.g. written by cdct_cnn_select), at most
 * max_count (0..n_regions) entries are used, and numbers outside the image
 * set are skipped.  Only the listed regions' labels (and costs) are
 * written; the rest of `labels` is left as it was.  With cdct_cnn_select
 * this is the selector's fallback: the exhaustive search re-decides the
 * regions the network is unsure of. */
cdct_status cdct_rd_search_subset(cdct_rd rd, const cdct_image* in, const int32_t* q, int32_t n_q,
                                  int32_t kappa_num, int32_t kappa_log2_den, const int64_t* region_index,
                                  const int64_t* count, int64_t max_count, uint8_t* labels,
                                  uint64_t* partition_cost, void* stream);

/* Code every region with a given quadtree (labels device [n_q][n_regions],
 * each < 17; a larger value is read as 0) and report, per step and region,
 * with the definitions of cdct_rd_search:
 *   cost  device [n_q][n_regions][2] uint64: J' of that partition (low, high)
 *   dist  device [n_q][n_regions][2] uint64: its distortion on the J' scale,
 *         sum over its blocks of (32 / N)^4 D = 2^24 32^4 SSE, or NULL
 *   bits  device [n_q][n_regions] int32: its rate R including the split
 *         flags, or NULL
 * Only the transform sizes the partition uses are computed.  This is the
 * encoder's final pass after a size decision, by the search or the network. */
cdct_status cdct_rd_evaluate(cdct_rd rd, const cdct_image* in, const int32_t* q, int32_t n_q, int32_t kappa_num,
                             int32_t kappa_log2_den, const uint8_t* labels, uint64_t* cost, uint64_t* dist,
                             int32_t* bits, void* stream);

/* ---- Learned quadtree selector (a small CNN) ---------------------------
 *
 * The paper's codec experiment (Sec. 6.2) leaves the transform-size choice
 * to the encoder; cdct_rd_search makes it by trying all 17 quadtrees.  This
 * network proposes the quadtree instead, from the region's pixels and the
 * quantiser slot; it is trained on the search's own labels (and, optionally,
 * its partition costs), and the search stays available as fallback and judge.
 * The network is the library's, not the paper's:
 *   a0 = x / 64 (x the region's pixels, 32 x 32, edge-replicated as for
 *        cdct_rd_search);
 *   a_l = maxpool2x2(relu(conv3x3(a_{l-1}, W_l) + b_l)), l = 1, 2, 3, with
 *        zero padding, channels 1 -> 16 -> 32 -> 32, sizes 32 -> 16 -> 8 -> 4;
 *   h = a_3 flattened in (y, x, channel) order (512 values);  u = Wf1 h;
 *   for quantiser slot k (0..3, a one-hot input):
 *        g = relu(u + bf1 + Wq[:, k]),  logits = Wf2 g + bf2 (17 labels, the
 *        label numbering of cdct_rd_search); the label is the first maximum.
 * Precision: weights (W_l, Wf1, Wq, Wf2) are used as bfloat16 copies (round
 * to nearest even) of float32 master weights; biases stay float32; every
 * stored activation (a_l, g) is bfloat16; products accumulate in float32 on
 * the tensor cores (the order of the sums is not fixed).
 *
 * Parameters: one float32 vector of CDCT_CNN_PARAMS values, in this order:
 *   W1 [16][3][3][1]   b1 [16]   W2 [32][3][3][16]  b2 [32]
 *   W3 [32][3][3][32]  b3 [32]   Wf1 [64][512]      Wq [64][4]   bf1 [64]
 *   Wf2 [17][64]       bf2 [17]
 * (W_l[o][dy][dx][i] multiplies a_{l-1}[y + dy - 1][x + dx - 1][i]).  The
 * caller owns every buffer (device memory) and initialises the weights. */
#define CDCT_CNN_PARAMS 48241
#define CDCT_CNN_LABELS 17
#define CDCT_CNN_SLOTS 4

/* Bytes of the packed inference weights (a multiple of 256). */
size_t cdct_cnn_packed_bytes(void);

/* params (device, CDCT_CNN_PARAMS floats) -> packed (device,
 * cdct_cnn_packed_bytes(), 16-byte aligned): the bfloat16 weights in the
 * layouts the inference kernel reads.  Re-run after every weight update. */
cdct_status cdct_cnn_pack(const float* params, void* packed, void* stream);

/* Proposed labels of every 32 x 32 region of `in` (regions numbered as for
 * cdct_rd_search) for n_slots (1..4) quantiser slots (host array, each
 * 0..3).  One fused launch.  Outputs (device):
 *   labels  [n_slots][n_regions] uint8 (required)
 *   logits  [n_slots][n_regions][17] float, or NULL
 *   margin  [n_slots][n_regions] float: best minus second-best logit (the
 *           selector's confidence; 0 on ties), or NULL
 * CDCT_EINVAL for 2^31 or more regions in one call (split the batch).  A
 * tensor-core wait that runs out is reported by cdct_check_device
 * (CDCT_ETIMEOUT); the outputs of that call are then incomplete. */
cdct_status cdct_cnn_infer(const void* packed, const cdct_image* in, const int32_t* slots, int32_t n_slots,
                           uint8_t* labels, float* logits, float* margin, void* stream);

/* Regions the selector is unsure of: every region whose smallest margin
 * over the n_slots slots (margin device [n_slots][n_regions], as written by
 * cdct_cnn_infer) is below `threshold`.  Their numbers go to region_index
 * (device int64, room for n_regions) in no particular order and their count
 * to *count (device int64, reset by the call).  Feed both to
 * cdct_rd_search_subset. */
cdct_status cdct_cnn_select(const float* margin, int64_t n_regions, int32_t n_slots, float threshold,
                            int64_t* region_index, int64_t* count, void* stream);

/* Device workspace of cdct_cnn_grad for `batch` regions (batch a positive
 * multiple of 64). */
cdct_status cdct_cnn_workspace_size(int32_t batch, size_t* bytes);

/* Loss and gradient of one batch, no update.
 *   regions   device int16 [batch][32][32], pixels in [-255, 255]
 *   slots     host [n_slots] (1..4 slots, each 0..3)
 *   labels    device uint8 [n_slots][batch], each < 17 (targets)
 *   partition_cost  device uint64 [n_slots][batch][17][2]: the 17
 *             partition costs J' per sample as cdct_rd_search writes them,
 *             or NULL (then mu is ignored); they give the normalised regret
 *             c_j = (J_j - J_min) / J_min (evaluated in double precision)
 *   grad      device float [CDCT_CNN_PARAMS] (overwritten)
 *   loss      device float [1]: mean over the batch x n_slots samples of
 *             -log p_label + mu sum_j p_j c_j, p = softmax(logits)
 *   workspace device, cdct_cnn_workspace_size() bytes, 256-byte aligned.
 * The forward pass repeats the inference arithmetic layer by layer; the
 * backward pass rounds du, dh and the input gradients of conv3 and conv2 to
 * bfloat16 before each product, treats every rounding as the identity, and
 * sends a max pool's gradient to the first maximum of its window (raster
 * order).  Weight gradients are reduced in a fixed order: the result is
 * reproducible bit for bit. */
cdct_status cdct_cnn_grad(const float* params, const int16_t* regions, int32_t batch, const int32_t* slots,
                          int32_t n_slots, const uint8_t* labels, const uint64_t* partition_cost, float mu,
                          float* grad, float* loss, void* workspace, size_t workspace_bytes, void* stream);

/* One Adam step (Kingma and Ba, 2015) in place on params, with state m, v
 * (device, CDCT_CNN_PARAMS floats each, zero before step 1) and step >= 1:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   params -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
cdct_status cdct_cnn_adam(float* params, const float* grad, float* m, float* v, int32_t step, float lr,
                          float beta1, float beta2, float eps, void* stream);

/* Synchronise `stream` and report whether a kernel of this library gave up
 * a bounded wait on the current device since the last check (the fused
 * kernel waits, with a time limit of about one second, for the bulk copies
 * that stage its input; the training GEMMs wait as long for their tensor-core
 * products).  Returns CDCT_ETIMEOUT and clears the record if so,
 * CDCT_OK otherwise.  Outputs of a call that timed out are incomplete. */
cdct_status cdct_check_device(void* stream);

/* Failure-detection test hook; the paper has no counterpart.  Makes the
 * library's bounded waits run out on purpose, with no GPU fault and nothing
 * left in flight, so that a test can check that the time-out is detected and
 * reported (cdct_check_device) and that the next calls work normally.
 *   mode 0: off (the default; normal one-second limits).
 *   bit 0: the fused pipelined kernel arms its staging barriers but issues no
 *          bulk copy, so every stage wait gives up after `wait_limit_cycles`
 *          SM cycles; its outputs are then not written.
 *   bit 1: the training GEMMs issue no tensor-core MMA and no commit, so
 *          their accumulator wait gives up after `wait_limit_cycles`.
 * `wait_limit_cycles` must lie in [1000, 2^31] when mode != 0 (ignored
 * otherwise).  The setting is process-wide and applies to launches made after
 * the call; CDCT_EINVAL for an invalid mode or limit. */
cdct_status cdct_set_fault_injection(int mode, int64_t wait_limit_cycles);

/* Host copy of a plan matrix (CDCT_MATRIX_*), computed by running the
 * library's own butterflies on unit vectors.  `out` is host memory of N*N
 * doubles (N for CDCT_MATRIX_S). */
cdct_status cdct_matrix(cdct_plan plan, int which, double* out);

/* Message of the last failed call on this thread ("" if none). */
const char* cdct_last_error(void);

/* Library version string. */
const char* cdct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CDCT_H */
