/*
 * litho.h - C ABI of the GB300 SOCS lithography imaging library (liblitho.so).
 *
 * The library evaluates, on one NVIDIA GB300 (sm_103a):
 *   - partially coherent aerial images in sum-of-coherent-systems (SOCS) form,
 *     I(x) = D * sum_k lam_k |(phi_k (x) m)(x)|^2, over K TCC eigen-kernels and
 *     several focus planes (paper Section III.A, Eqs. (1)-(4));
 *   - the Gaussian-blur + threshold resist (Eq. (5));
 *   - exact area-coverage rasterisation of rectangle masks;
 *   - marching-squares contours of the resist image and the edge-placement
 *     error at target control points, through focus (Section II.D, Eqs. (6)-(8));
 *   - the ILT mask gradient through the resist and imaging (the adjoint of the
 *     above; pixel-based ILT is the paper's Section I prior art), and the
 *     intensity vector-Jacobian product on its own;
 *   - the AI initialiser's input channels and print-consistency images
 *     (Eqs. (9), (15)-(17));
 *   - a continuous-batching request server over all of it.
 * The image, its resist, the ILT gradient, the VJP and the AI channels can be
 * evaluated on a coarse grid of at least 2C points (LITHO_GRID_COARSE) with
 * an exact Fourier interpolation to N: the same results up to FP32 rounding.
 *
 * Conventions shared by every entry point:
 *   - Grids are N x N, row-major, x fastest; pixel size in nm at the wafer.
 *   - Frequencies f_u = u / (N * pixel), u in [-N/2, N/2).  Kernels live on a
 *     C x C crop centred on DC, crop index c <-> u = c - C/2 (C a multiple of
 *     32, C/2 above the band radius (1 + sigma_max) NA / wavelength).
 *   - The mask spectrum is M(u) = N^-2 * DFT(m)(u): a clear mask (m = 1)
 *     images to I = dose everywhere with the full-rank kernel set.
 *   - Device pointers (suffix _dev) are CUDA global memory owned by the caller
 *     (for example torch tensors); host pointers (suffix _host) are plain CPU
 *     memory, pinned or pageable.  Handles (litho_kernels, litho_server) and the
 *     memory they reference are owned by the library.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Device work is enqueued on it and the call returns without
 *     waiting, unless a host output (loss_host, *_host buffers) is requested.
 *   - No C++ exception crosses this boundary.  Every call returns a
 *     litho_status; on failure litho_last_error() gives a message (per thread).
 *   - Nothing here allocates device memory except litho_make_kernels /
 *     litho_upload_kernels (the kernel handle) and the server.  Scratch is the
 *     caller's `workspace`, sized by the *_workspace_size queries.
 */
#ifndef LITHO_H
#define LITHO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LITHO_OK = 0,
  LITHO_EINVAL = 1,       /* bad argument (size, null pointer, alignment, mismatch) */
  LITHO_ENOMEM = 2,       /* host or device allocation failed, or workspace too small */
  LITHO_ECUDA = 3,        /* a CUDA call failed; message in litho_last_error() */
  LITHO_EBUSY = 4,        /* server queue full */
  LITHO_ETIMEOUT = 5,     /* poll timed out, or a device-side wait gave up */
  LITHO_ECANCELED = 6,    /* request cancelled */
  LITHO_EUNSUPPORTED = 7  /* valid request this build or device does not implement */
} litho_status;

typedef enum {
  LITHO_SRC_ANNULAR = 0,     /* sigma_in <= |sigma| <= sigma_out */
  LITHO_SRC_QUADRUPOLE = 1,  /* four discs, radius pole_radius, centred on the x/y axes at pole_sigma */
  LITHO_SRC_CUSTOM = 2       /* weights custom_w on the src_grid x src_grid lattice */
} litho_source_kind;

/* Illumination and projection optics (paper Eq. (2): source S and pupil P).
 * The source is sampled on the lattice sigma = (i/h, j/h), i, j in [-h, h],
 * h = (src_grid - 1)/2, in units of NA/wavelength; membership tests are
 * inclusive.  Weights are equal (annular, quadrupole) or custom_w, and are
 * normalised to sum 1.  The pupil is scalar and aberration-free with the NA
 * cut-off and a defocus phase exp(i 2 pi z (sqrt((n/l)^2 - f^2) - n/l)). */
typedef struct {
  double wavelength_nm;   /* 193 (ArF immersion) or 13.5 (EUV) */
  double na;              /* numerical aperture, 0 < NA <= n_medium */
  double n_medium;        /* immersion index (1.44 ArF immersion, 1 EUV) */
  int kind;               /* litho_source_kind */
  int src_grid;           /* odd, >= 3 */
  double sigma_in, sigma_out;        /* annular */
  double pole_sigma, pole_radius;    /* quadrupole */
  const double* custom_w; /* CUSTOM: src_grid*src_grid weights, row j (y) major; copied */
} litho_optics;

typedef enum {
  LITHO_PREC_FFT32 = 0,  /* FP32 FFT path (band multiply + two inverse FFT passes) */
  LITHO_PREC_BF16 = 1,   /* tcgen05 DFT-GEMM, bf16 operands, FP32 accumulation */
  LITHO_PREC_BF16X3 = 2, /* tcgen05 DFT-GEMM, split bf16 hi/lo, three products */
  LITHO_PREC_FP16X3 = 3, /* tcgen05 DFT-GEMM, split fp16 hi/lo (scaled), three products */
  LITHO_PREC_FP16 = 4    /* tcgen05 DFT-GEMM, fp16 operands (scaled), FP32 accumulation */
} litho_precision;
/* OR-ed into a precision: evaluate the coherent fields on the coarse grid
 * nc x nc, nc >= 2C (litho_kernels_grid: the smallest power of two, or 896 =
 * 16 x 8 x 7 for the tensor-core path), and interpolate I to N x N
 * exactly (I = sum_k lam_k |E_k|^2 has no frequency at or beyond C along
 * either axis, so nc >= 2C samples determine it; the interpolation is a
 * forward transform on nc and an inverse transform on N).  Ignored when
 * nc >= N.  Exact up to rounding; saves about (N/nc)^2 of the stage-2 work. */
#define LITHO_GRID_COARSE 0x100
/* Tensor-core modes need n a multiple of 128 and an sm_103 device (else
 * EUNSUPPORTED); the fp16 modes scale the stage-1 fields per kernel by a power
 * of two chosen for masks with |m| <= 1. */

typedef struct litho_kernels litho_kernels; /* device-resident SOCS kernels for one (optics, N, pixel, focus list, K) */
typedef struct litho_server litho_server;

/* ---- kernels (paper Eqs. (2)-(3)) ------------------------------------------------------- */

/* Builds the top-k TCC eigen-kernels of every focus plane on the host in FP64
 * (TCC = A A^H with A[u,s] = sqrt(w_s) P(f_u + sigma_s; z); eigenpairs from the
 * Gram matrix A^H A) and uploads them.  k larger than the TCC rank gives zero
 * kernels (lam = 0) for the excess modes; the rank is reported by
 * litho_kernels_info.  n must be a power of two in [16, 2048].
 * Errors: EINVAL (bad optics/sizes), ENOMEM, ECUDA. */
litho_status litho_make_kernels(const litho_optics* optics, int n, double pixel_nm, const double* defocus_nm,
                                int n_focus, int k, litho_kernels** out);

/* The FP64 host half of litho_make_kernels for one focus plane, with no GPU
 * involved: call with phi_host = NULL to learn *crop, then again with
 * lambda_host of k doubles and phi_host of k*crop*crop*2 doubles ([k][v][u],
 * re/im interleaved).  rank, trace, gap as in litho_kernels_info; any of the
 * scalar outputs may be NULL. */
litho_status litho_tcc_kernels_host(const litho_optics* optics, int n, double pixel_nm, double defocus_nm, int k,
                                    int* crop, double* lambda_host, double* phi_host, int* rank, double* trace,
                                    double* gap);

/* Wraps caller-supplied kernels: lambda_host[n_focus*k] (>= 0) and
 * phi_host[n_focus][k][crop][crop][2] (re, im interleaved), crop a multiple of
 * 32 in [32, n].  Used to image with kernels from another source (for example
 * a reference implementation) through the same device path.  Copies the data. */
litho_status litho_upload_kernels(int n, double pixel_nm, int n_focus, int k, int crop, const double* lambda_host,
                                  const double* phi_host, litho_kernels** out);

/* Describes a kernel set.  Any output pointer may be NULL.  rank_host,
 * trace_host and gap_host have n_focus entries, lambda_host n_focus*k.
 * gap = lam_k - lam_{k+1} of the built TCC (0 for uploaded kernels); a gap
 * below 1e-12 * lam_1 means the cut at k splits a degenerate cluster. */
litho_status litho_kernels_info(const litho_kernels* h, int* n, int* crop, int* n_focus, int* k, int* rank_host,
                                double* lambda_host, double* trace_host, double* gap_host);

/* The coarse evaluation grids LITHO_GRID_COARSE uses (the image has no
 * frequency at or beyond crop, so 2 crop samples per axis determine it
 * exactly): *nc_fft for LITHO_PREC_FFT32, the smallest power of two >= 2 crop;
 * *nc_tensor for the tensor-core precisions, the same or 896 = 16 x 8 x 7 when
 * 2 crop <= 896 is smaller.  0 when the grid is not below n (the flag is then
 * ignored for that path).  Either output may be NULL. */
litho_status litho_kernels_grid(const litho_kernels* h, int* nc_fft, int* nc_tensor);

/* Copies the FP64 kernels phi[n_focus][k][crop][crop][2] back to the host. */
litho_status litho_kernels_phi(const litho_kernels* h, double* phi_host);

void litho_free_kernels(litho_kernels* h);

/* ---- aerial image (paper Eq. (4)) ------------------------------------------------------------ */

/* Bytes of device scratch litho_aerial needs for a batch of b clips. */
litho_status litho_aerial_workspace_size(const litho_kernels* h, int b, litho_precision prec, size_t* bytes);

/* I[b][f][y][x] = dose * sum_k lam_fk |E_fk(x,y)|^2 for masks m[b][y][x]
 * (values in [0,1], any real values accepted).  mask_dev and intensity_dev are
 * float32 device arrays; workspace_dev must be 256-byte aligned and hold
 * litho_aerial_workspace_size bytes.  Asynchronous on `stream`.
 * Errors: EINVAL, ENOMEM (workspace too small), EUNSUPPORTED (precision not
 * available for this crop), ECUDA. */
litho_status litho_aerial(const litho_kernels* h, const float* mask_dev, int b, double dose, litho_precision prec,
                          float* intensity_dev, void* workspace_dev, size_t workspace_bytes, void* stream);

/* litho_aerial followed by litho_resist (paper Eqs. (4)-(5)) in one call:
 * intensity_dev as litho_aerial, iblur_dev[b][F][n][n] (f32) the periodic
 * Gaussian blur of every plane with sigma_nm (the kernel set's pixel size),
 * printed_dev (u8, may be NULL) = [iblur >= threshold].  Same workspace as
 * litho_aerial (litho_aerial_workspace_size).  With LITHO_GRID_COARSE (when it
 * applies) the blur is applied in the frequency domain during the exact
 * interpolation to n x n: the image spectrum is band-limited, so multiplying
 * it by the transfer function of the truncated taps, sum_a g[a]
 * e^{-2 pi i f a/n} in each axis, is the periodic convolution exactly (up to
 * rounding), and the image and its blur come out of one complex inverse
 * transform as its real and imaginary parts.  Otherwise the litho_resist
 * kernel runs after the image.  Errors: as litho_aerial and litho_resist. */
litho_status litho_aerial_resist(const litho_kernels* h, const float* mask_dev, int b, double dose,
                                 litho_precision prec, float* intensity_dev, double sigma_nm, double threshold,
                                 float* iblur_dev, uint8_t* printed_dev, void* workspace_dev, size_t workspace_bytes,
                                 void* stream);

/* Waits for `stream` and reports LITHO_ETIMEOUT if, since the last check, a
 * tensor-core kernel of this kernel set gave up waiting on one of its
 * pipeline barriers (each such wait is bounded at about two seconds; the
 * kernel then drains its own copies, frees its tensor memory and returns,
 * leaving its output incomplete).  Clears the flag.  LITHO_OK otherwise. */
litho_status litho_check_device(const litho_kernels* h, void* stream);

/* Self-test of that mechanism, for failure-detection tests: launches one
 * block whose thread waits, with the same bounded wait the tensor-core
 * pipeline uses, on a barrier that nothing ever signals, limited to limit_ms
 * (0 < limit_ms <= 2000).  The wait gives up, records the error and the
 * kernel returns; the call then reports LITHO_ETIMEOUT through
 * litho_check_device (which also clears the flag).  The device stays usable.
 * Any other status means the limit did not work. */
litho_status litho_selftest_wait_limit(const litho_kernels* h, double limit_ms, void* stream);

/* The same computation from host memory, optionally followed by the resist:
 * copies mask_host[b][n][n] in, images, and copies back whichever of
 * intensity_host[b][F][n][n] (f32) and printed_host[b][F][n][n] (u8, the
 * litho_resist threshold of the blurred image with sigma_nm and threshold) is
 * non-NULL, then waits for the stream.  Device buffers are carved from
 * workspace_dev (litho_aerial_host_workspace_size bytes).  Batches of 4 or more
 * clips run in chunks on three library streams (ordered after `stream`):
 * input copies, the kernels of one chunk after another, and output copies,
 * so that neighbouring chunks' copies overlap the kernels; pinned host
 * memory lets the copies run asynchronously at full link speed.  Calls on
 * the same kernel set are serialised. */
litho_status litho_aerial_host_workspace_size(const litho_kernels* h, int b, litho_precision prec, size_t* bytes);
litho_status litho_aerial_host(const litho_kernels* h, const float* mask_host, int b, double dose,
                               litho_precision prec, float* intensity_host, double sigma_nm, double threshold,
                               uint8_t* printed_host, void* workspace_dev, size_t workspace_bytes, void* stream);
/* Host timestamps of the last completed litho_aerial_host call (any thread):
 * event i has tag tags[i] and happened ms[i] milliseconds after the call
 * began.  Tags: 8 c + 0 / 1 / 2 when chunk c's input copy, its kernels and
 * its output copies had been enqueued; -1 when all work was enqueued and
 * the final wait began; -2 when the wait ended; and, in device time since
 * the call's first work item started, 100 + 8 c + 0 / 1 / 2 when chunk c's
 * input copy, its kernels and its output copies finished (CUDA events).  Up
 * to max_events are written; *count receives the number the call recorded.
 * A host-side stall shows as a late enqueue, a device-side one as a long
 * wait, and the device times tell copies from kernels. */
litho_status litho_host_trace_read(int max_events, int* tags, double* ms, int* count);

/* The FP32 aerial image (same result as litho_aerial with LITHO_PREC_FFT32)
 * without any device allocation and without a workspace argument.  The paper
 * has no counterpart: this exists for callers that cannot allocate device
 * memory when they call in, such as a host application that owns all device
 * memory through its own pool, or a latency-critical loop that cannot take
 * the device-wide stall cudaMalloc/cudaFree may cause.
 * Scratch lives in one fixed library array of litho_aerial_noalloc_max_bytes()
 * bytes (32 MiB) that every GPU loading the library reserves until exit.
 * Clips are imaged one after another; the scratch one clip needs (row and
 * crop spectra plus n_focus*k stage-1 fields, about 8*N*C*(1 + n_focus*k)
 * bytes) must fit, else EINVAL with the sizes in the message (for example
 * N = 256 with 8 kernels fits; N = 2048 with 72 kernel planes does not).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and each call
 * overwrites what the previous one left: calls that can run at the same time
 * on the GPU (different streams, or different host threads) race and corrupt
 * each other's results; serialise them on one stream.  The kernel set's
 * device must be the current device (else EINVAL: the scratch address is
 * per device).  mask_dev and intensity_dev must be 16-byte aligned and the
 * dose finite (else EINVAL), as for litho_aerial.  Asynchronous on
 * `stream`. */
litho_status litho_aerial_noalloc(const litho_kernels* h, const float* mask_dev, int b, double dose,
                                  float* intensity_dev, void* stream);
size_t litho_aerial_noalloc_max_bytes(void);

/* ---- resist (paper Eq. (5)) ------------------------------------------------------------------- */

/* iblur = g (x) I with the periodic separable Gaussian g[j] ~ exp(-(j p)^2 / (2 s^2)),
 * |j| <= ceil(4 s / p), sum g = 1; printed = (iblur >= threshold) as 0/1 bytes.
 * `planes` independent n x n planes.  printed_dev may be NULL.  The blur
 * radius must be below n/2. */
litho_status litho_resist(const float* intensity_dev, int planes, int n, double pixel_nm, double sigma_nm,
                          double threshold, float* iblur_dev, uint8_t* printed_dev, void* stream);

/* ---- gradients of the image and the AI initialiser's inputs (paper Eqs. (9), (15)-(17)) ---------- */

/* Vector-Jacobian product of Eq. (4): dm[c][x'] = sum over the planes f in
 * [f_first, f_first + f_count) of sum_x q[c][f][x] dI_f(x)/dm(x') for masks
 * mask[c] (f32 [b][n][n]), with q = upstream_dev[b][n_focus][n][n] (the
 * planes outside the range are not read) or, when upstream_dev is NULL, 1 on
 * every pixel (the gradient of the total intensity).  The same adjoint as
 * litho_ilt_grad without the resist and sigmoid factors: 2 D N^-2 Re IDFT of
 * sum_k lam_k conj(Phi_k) DFT_crop(q E_k).  With q = 1 this sum is, by
 * Parseval, N^2 sum_k lam_k |Phi_k|^2 Mhat (Mhat the mask's crop spectrum), which
 * is what is evaluated then (no field is transformed; the grid flag has no
 * effect on the result).  Workspace as litho_ilt_workspace_size
 * (the smaller size evaluates one plane of one clip at a time).  prec:
 * LITHO_PREC_FFT32 (else EUNSUPPORTED), optionally | LITHO_GRID_COARSE (the
 * fields and the adjoint on the coarse grid, q low-passed to the image band
 * and sampled there: the full-grid result up to FP32 rounding).  Async. */
litho_status litho_intensity_vjp_workspace_size(const litho_kernels* h, int b, size_t* full_bytes, size_t* min_bytes);
litho_status litho_intensity_vjp(const litho_kernels* h, const float* mask_dev, int b, double dose,
                                 litho_precision prec, int f_first, int f_count, const float* upstream_dev,
                                 float* dm_dev, void* workspace_dev, size_t workspace_bytes, void* stream);

/* Eq. (9): the three input channels of the AI initialiser for binary targets
 * Z_t = target[b][n][n] (0/1 f32): x[c][0] = Z_t, x[c][1] = I0 / max I0 with I0
 * the aerial image of the target at plane `focus`, x[c][2] = (g - min g) /
 * (max g - min g) with g the gradient of that plane's total intensity with
 * respect to the mask (litho_intensity_vjp of ones), the extremes taken over
 * the batch (a constant channel becomes 0).  x is f32 [b][3][n][n], 1 <= b <=
 * 65535.  Workspace: litho_ai_inputs_workspace_size(h, b) bytes, 256-byte
 * aligned.  prec:
 * LITHO_PREC_FFT32 (else EUNSUPPORTED), optionally | LITHO_GRID_COARSE (fields
 * and adjoint on the coarse grid, the image interpolated exactly: the same
 * channels up to FP32 rounding).  Both channels come from one evaluation of
 * the stage-1 fields per group of clips.  Async. */
litho_status litho_ai_inputs_workspace_size(const litho_kernels* h, int b, size_t* bytes);
litho_status litho_ai_inputs(const litho_kernels* h, const float* target_dev, int b, double dose, int focus,
                             litho_precision prec, float* x_dev, void* workspace_dev, size_t workspace_bytes,
                             void* stream);

/* Eqs. (15)-(17): z_round = [G (x) Z_t >= tau_round] with G the periodic,
 * normalised Gaussian of sigma_round_nm truncated at 4 sigma (as
 * litho_resist), z_print = [I >= tau_print] on the images intensity[b][n][n],
 * and, when loss_dev is not NULL, loss[c] = sum |z_print - z_round| (int64, the
 * number of pixels where the two differ).  blur_dev (f32 [b][n][n]) receives
 * G (x) Z_t.  n a multiple of 32; z_round_dev and z_print_dev 16-byte
 * aligned.  Async. */
litho_status litho_print_images(const float* target_dev, const float* intensity_dev, int b, int n, double pixel_nm,
                                double sigma_round_nm, double tau_round, double tau_print, uint8_t* z_round_dev,
                                uint8_t* z_print_dev, int64_t* loss_dev, float* blur_dev, void* stream);

/* ---- rectangle masks to grey levels (the object m of Eq. (1)) --------------------------------- */

/* Area-coverage rasterisation: mask[c][i][j] = area of the union of clip c's
 * rectangles inside pixel [j, j+1) x [i, i+1) (pixel units, x = column,
 * y = row), periodic with period n, overlapping rectangles counted once; so
 * shapes off the pixel grid become exact grey levels instead of centre
 * samples (exact up to FP32 rounding).  Rectangles rects_dev[4 r .. 4 r + 3] =
 * (x0, y0, x1, y1) (f32, 16-byte aligned), clip c owning r in
 * [rect_start[c], rect_start[c+1]) (int64, device); max_rects bounds any one
 * clip's count, max_side_px every side (0 < x1 - x0 <= max_side_px, same in
 * y); a clip with more rectangles or one outside those bounds gets an all-NaN
 * mask.  n a multiple
 * of 16.  Workspace: litho_rasterize_workspace_size bytes (it holds the
 * rectangles' tile lists, (ceil(max_side_px/16) + 5)^2 entries of 16 bytes per
 * rectangle), 256-byte aligned.  Asynchronous (five launches).  Errors: EINVAL,
 * ENOMEM (workspace too small), ECUDA. */
litho_status litho_rasterize_workspace_size(int b, int n, int64_t max_rects, int max_side_px, size_t* bytes);
litho_status litho_rasterize(const float* rects_dev, const int64_t* rect_start_dev, int b, int64_t max_rects,
                             int max_side_px, int n, float* mask_dev, void* workspace_dev, size_t workspace_bytes,
                             void* stream);

/* ---- contours and edge placement (paper section II.D, Eqs. (6)-(8)) ----------------------------- */

/* Marching-squares contours of `planes` resist images iblur[p][n][n] (f32) at
 * `threshold` (compared in FP32).  Cell (i, j) has the corners TL = I[i][j],
 * TR = I[i][j+1], BR = I[i+1][j+1], BL = I[i+1][j] (periodic); a corner is
 * inside (printed) when I >= T.  A cell edge whose corners differ is crossed
 * at the linear interpolation of I - T; a saddle (only TL and BR, or only TR
 * and BL, inside) joins its inside corners when ((TL + TR) + (BR + BL))/4 >= T
 * and separates them otherwise.  Each segment is oriented so that the corner
 * it cuts off lies on its left when inside and on its right when outside, and
 * a segment between opposite edges has the inside pair on its left (left of
 * p0 -> p1: cross(p1 - p0, q - p0) > 0): closed contours chain end to start
 * with the printed region on the left.
 * Output, deterministic: segment s = (x0, y0, x1, y1) in pixels (x = column,
 * y = row, absolute cell coordinates in FP32, so a cell of the last row or
 * column can reach n) at seg_dev[4 s .. 4 s + 3], its cell i n + j at cell_dev[s] (may be
 * NULL); segments in plane order, cells row-major, the two of a saddle by
 * their start edge (0 top, 1 right, 2 bottom, 3 left).  plane_start_dev
 * [planes + 1] (int64) receives the index of each plane's first segment and
 * the total; segments at or beyond `capacity` are counted but not written,
 * so a caller that sees total > capacity calls again with more room.
 * Workspace: litho_contours_workspace_size bytes, 256-byte aligned; seg_dev
 * 16-byte aligned.  Asynchronous on `stream` (four launches).  Errors:
 * EINVAL, ENOMEM (workspace too small), ECUDA. */
litho_status litho_contours_workspace_size(int planes, int n, size_t* bytes);
litho_status litho_contours(const float* iblur_dev, int planes, int n, double threshold, float* seg_dev,
                            int32_t* cell_dev, int64_t capacity, int64_t* plane_start_dev, void* workspace_dev,
                            size_t workspace_bytes, void* stream);

/* Edge-placement error, Eq. (6), at m control points on target edges:
 * epe[p][k] = -(I_b(r_k) - T) / |grad I_b(r_k)| in nm for every plane p, with
 * the target's value at its own edge read as the threshold T, r_k =
 * (points[2k], points[2k+1]) = (x, y) in pixels (f32), I_b and its gradient
 * interpolated bilinearly from the pixels and from their periodic central
 * differences, the gradient per nm (divided by pixel_nm).  NaN where the
 * gradient vanishes.  Asynchronous. */
litho_status litho_epe(const float* iblur_dev, int planes, int n, double pixel_nm, double threshold,
                       const float* points_dev, int m, float* epe_dev, void* stream);

/* litho_epe for a batch of clips in one launch: the points of clip c are
 * points[start[c] .. start[c+1]) (start_dev: clips + 1 int64 on the device,
 * start[0] = 0, non-decreasing, start[clips] = m_total; empty clips allowed)
 * and are evaluated on that clip's planes iblur[c][0 .. planes) (f32
 * [clips][planes][n][n]); epe[p][k] for all m_total points, plane-major, so
 * that one litho_epe_through_focus call covers the batch.  Each value equals
 * litho_epe on the clip alone.  A start array that breaks these rules gives
 * wrong values but no access outside the buffers.  Asynchronous. */
litho_status litho_epe_batch(const float* iblur_dev, int clips, int planes, int n, double pixel_nm, double threshold,
                             const float* points_dev, const int64_t* start_dev, int64_t m_total, float* epe_dev,
                             void* stream);

/* Eqs. (7)-(8) from epe[planes][m]: avg[k] = mean of the on-focus plane f0 and
 * the defocused planes fp and fn; eff[k] = e0 - tol_pos if e0 > tol_pos,
 * e0 - tol_neg if e0 < tol_neg, else avg[k] (e0 = epe[f0][k]; a value equal to
 * a tolerance takes the average).  Either output may be NULL.  Asynchronous. */
litho_status litho_epe_through_focus(const float* epe_dev, int planes, int m, int f0, int fp, int fn, double tol_neg,
                                     double tol_pos, float* avg_dev, float* eff_dev, void* stream);

/* ---- ILT gradient -------------------------------------------------------------------------------- */

/* Workspace for litho_ilt_grad: `full_bytes` keeps every focus plane's
 * stage-1 fields for the backward pass; `min_bytes` keeps one focus plane at a
 * time and recomputes it in the backward pass. */
litho_status litho_ilt_workspace_size(const litho_kernels* h, int b, size_t* full_bytes, size_t* min_bytes);

/* Loss and gradient of ILT over all focus planes of h, per clip:
 *   m = sigmoid(mask_steep * theta), I_f = dose * SOCS_f(m), Ib_f = g (x) I_f,
 *   Z_f = sigmoid(resist_steep * (Ib_f - threshold)),
 *   loss = sum_f sum_x (Z_f - target)^2,   grad = d loss / d theta.
 * theta_dev, target_dev, grad_dev: float32 [b][n][n] on the device (theta_dev
 * 16-byte aligned, else EINVAL).
 * loss_host (may be NULL): b doubles, reduced in FP64 on the device; when
 * given, the call waits for the stream.  With the full workspace each clip's
 * loss and gradient are bit-identical whatever the number of clips in the
 * call: the partial sums follow a partition fixed per clip (per row pair of
 * each plane on the coarse grid).  A workspace between min_bytes and
 * full_bytes selects recomputation of the forward fields; below min_bytes is
 * ENOMEM.  prec: LITHO_PREC_FFT32 (else EUNSUPPORTED), optionally with
 * LITHO_GRID_COARSE: the fields, the image and the adjoint transforms are
 * evaluated on the coarse grid of litho_kernels_grid (when it is below n),
 * the image is interpolated exactly to n for the resist and the loss, and
 * d loss / dI is low-passed to the image band (2C) and sampled on that grid
 * before the adjoint; the products with the fields are cropped to the field
 * band, where nothing aliases on a grid of at least 2C points, so the
 * gradient is the full-grid one up to FP32 rounding. */
litho_status litho_ilt_grad(const litho_kernels* h, const float* theta_dev, const float* target_dev, int b,
                            double dose, double mask_steep, double resist_steep, double threshold, double sigma_nm,
                            litho_precision prec, float* grad_dev, double* loss_host, void* workspace_dev,
                            size_t workspace_bytes, void* stream);

/* ---- serving ------------------------------------------------------------------------------------- */

typedef enum { LITHO_REQ_IMAGE = 0, LITHO_REQ_ILT_STEP = 1 } litho_request_kind;

/* One request: a single clip.  All pointers are host memory that must stay
 * valid until the request completes (poll returns OK/ECANCELED).
 *   IMAGE:    input = mask[n][n] -> output = I[n][n] at defocus_nm.
 *   ILT_STEP: input = theta[n][n], target[n][n] -> output = grad[n][n], *loss. */
typedef struct {
  int kind;                 /* litho_request_kind */
  litho_optics optics;
  int n;
  double pixel_nm;
  double defocus_nm;
  int k;
  int precision;            /* litho_precision (ILT steps use FFT32) */
  double dose;
  double sigma_nm, threshold, mask_steep, resist_steep;   /* ILT step */
  const float* input_host;
  const float* target_host;
  float* output_host;
  double* loss_host;
} litho_request;

typedef struct {
  uint64_t submitted, completed, rejected, cancelled;
  double p50_ms, p99_ms;          /* submit -> completion latency over completed requests */
  double mpx_per_s;               /* completed pixels / (last completion - first submit) */
  size_t hbm_high_water;          /* peak bytes of admitted work */
  int kernel_sets_cached;
  uint64_t batches;               /* batches launched (completed / batches = mean clips per batch) */
  int max_batch;                  /* clips in the largest batch */
} litho_serve_stats_t;

/* A server with its own scheduler thread, max_slots concurrent batches (one
 * CUDA stream each), admission while the summed device footprint of running
 * batches stays within hbm_budget_bytes, and a queue of max_queue waiting
 * requests.  Continuous batching: when a slot frees, the oldest request that
 * fits takes with it the queued requests that can share its launches (the
 * same optics, n, pixel, focus, k, kind, precision, dose and ILT constants),
 * in arrival order, up to 64 clips and 8 x 2048^2 pixels of work (an ILT
 * step counting twice), and the batch runs as one grouped
 * litho_aerial / litho_ilt_grad call; each request's result is the same,
 * bit for bit, as the request run alone.  Kernel sets are built once per
 * (optics, n, pixel, focus, k) and stay resident (the paper's GPU-residency
 * principle, its Section II.D).  Batches take their device memory from the
 * device's default memory pool, in which the server reserves its budget (at
 * most half of the free memory) when it is created and which it trims when it
 * is destroyed. */
litho_status litho_serve_create(size_t hbm_budget_bytes, int max_slots, int max_queue, litho_server** out);
/* EBUSY if the queue is full; EINVAL if the request's footprint exceeds the
 * whole budget or its fields are invalid. */
litho_status litho_serve_submit(litho_server* s, const litho_request* req, uint64_t* ticket);
/* OK when done (output written), ECANCELED, ETIMEOUT if still pending after
 * timeout_ms (0 = just check), EINVAL for an unknown ticket, or the request's
 * own error status.  Never blocks longer than timeout_ms. */
litho_status litho_serve_poll(litho_server* s, uint64_t ticket, int timeout_ms);
/* Cancels a request that has not started; EBUSY if it is already running. */
litho_status litho_serve_cancel(litho_server* s, uint64_t ticket);
litho_status litho_serve_stats(litho_server* s, litho_serve_stats_t* out);
/* Starts a new statistics window (latencies, counters, throughput span,
 * high-water mark); queued and running requests and the kernel cache are
 * untouched.  Requests submitted before the reset that complete after it
 * still count as completed in the new window. */
litho_status litho_serve_stats_reset(litho_server* s);
/* Waits for running requests, cancels queued ones, frees everything. */
void litho_serve_destroy(litho_server* s);
/* Host-side fault injection for tests: bit 0 makes the next admitted
 * request's device allocation fail (the request ends with LITHO_ENOMEM and
 * the server carries on); bit 1 makes the next admitted request slow (a
 * fixed 200 ms device delay on its slot's stream before its work: one thread
 * spinning on the SM clock, which always ends), so that requests on the
 * other slots can be seen to complete meanwhile.  A request that takes an
 * injected fault runs alone (no batch).  No GPU fault is involved. */
litho_status litho_serve_inject_fault(litho_server* s, int fault_mask);

/* ---- tracing ------------------------------------------------------------------------------------- */

/* Per-stage device timing.  While enabled, every stage the library enqueues is
 * bracketed by CUDA events on its stream (stages: mask_spectrum, stage1_fft,
 * stage2_fft, stage1_gemm_operands, stage2_gemm, resist, ilt_forward,
 * ilt_backward, ilt_reduce, upsample, upsample_resist, contours, epe,
 * raster).  Every stage also opens an NVTX range of the same name on the
 * calling host thread, enabled or not (free unless an NVTX tool is attached).
 * litho_profile_read waits for the recorded events
 * and reports, for up to max_stages stages that ran since the last reset,
 * the name (32-byte slots in `names`), the summed device milliseconds and the
 * number of kernel launches; *count receives how many were written. */
litho_status litho_profile_enable(int on);
void litho_profile_reset(void);
litho_status litho_profile_read(int max_stages, char* names, double* total_ms, long long* launches, int* count);

/* ---- misc ----------------------------------------------------------------------------------------- */

const char* litho_last_error(void);
const char* litho_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LITHO_H */
