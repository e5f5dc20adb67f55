/*
 * supra.h -- C ABI of a B300-native (sm_103a) implementation of the real-time
 * processing chain of SUPRA (Goebl, Navab, Hennersperger, arXiv:1711.06127):
 * receive delay-and-sum beamforming of raw channel data, IQ demodulation and
 * envelope detection, log compression and 2D/3D scan conversion.
 *
 * Paper passages:
 *   Sec. 1, pipeline step list: receive beamforming -> RF, envelope detection,
 *       log-compression, scan conversion of lines that need not be parallel.
 *   Sec. 2, method list items 1-5: dynamic receive beamforming for a flexible
 *       scanline layout and multi-line acquisition; delay-and-sum of raw
 *       channel data after A/D conversion; envelope detection by IQ
 *       demodulation; log compression to a target dynamic range; scan
 *       conversion in 2D and 3D.
 *   Sec. 2: transmit parameters are computed once for a fixed acquisition --
 *       here supra_plan_create builds every geometry-dependent table once.
 *   Table 1: the four nodes Beamformer / Envelope / Log comp. / Scan conv.
 *       -- one entry point each, plus the fused chain supra_bmode.
 *
 * Units: metres, seconds, Hz.  Probe frame: the array lies in the z = 0 plane,
 * x lateral, y elevation, z depth.
 *
 * Conventions for every entry point:
 *   - Return 0 (SUPRA_OK) or a negative SUPRA_E* code; nothing is thrown.
 *   - Data pointers passed to compute entry points are caller-owned DEVICE
 *     pointers of the current CUDA device; `stream` is a cudaStream_t (NULL =
 *     legacy default stream).  Calls are asynchronous and stream-ordered; a
 *     SUPRA_ECUDA return reports a launch error seen at call time only.
 *   - Host arrays passed to supra_plan_create are copied; the caller may free
 *     them when it returns.
 *   - A plan is immutable after creation and may be used concurrently from
 *     several host threads and streams.
 *   - Device-side failures (a bounded wait that ran out, a staging window
 *     overflow) set a device status word read by supra_device_status().
 */
#ifndef SUPRA_H
#define SUPRA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SUPRA_API __attribute__((visibility("default")))
#else
#define SUPRA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define SUPRA_OK 0
#define SUPRA_EINVAL (-1)      /* bad argument, shape or parameter range         */
#define SUPRA_ENOMEM (-2)      /* device or host allocation failed               */
#define SUPRA_ECUDA (-3)       /* CUDA runtime error at call time                */
#define SUPRA_ETIMEOUT (-4)    /* a bounded device-side wait ran out             */
#define SUPRA_EINTERNAL (-5)   /* internal consistency check failed              */
#define SUPRA_EWORKSPACE (-6)  /* workspace missing, misaligned or too small     */

/* ---- apodization windows (evaluated at u = offset / half-aperture in [-1,1]) */
#define SUPRA_WINDOW_RECT 0    /* 1                                              */
#define SUPRA_WINDOW_HANN 1    /* (1 + cos(pi u)) / 2                            */
#define SUPRA_WINDOW_HAMMING 2 /* 0.54 + 0.46 cos(pi u)                          */

/* ---- scanline layouts known to scan conversion ---------------------------- */
#define SUPRA_GEOM_LINEAR 0    /* parallel lines along +z from evenly spaced x on z = 0            */
#define SUPRA_GEOM_SECTOR 1    /* lines in the xz plane from one apex at evenly spaced angles       */
#define SUPRA_GEOM_PYRAMID 2   /* lines from one apex along normalize(tan tx, tan ty, 1), tx and ty
                                  evenly spaced; line index = iy * lines_x + ix                     */

/* Probe: element positions, [n_el][3] doubles (host). */
typedef struct supra_probe {
    int32_t n_el;
    const double *elem_pos;
} supra_probe;

/* Transmit/receive scan geometry (Sec. 2 item 1: fully flexible scanline
 * layout; multi-line acquisition = several lines sharing a transmit event). */
typedef struct supra_scan {
    int32_t n_tx;               /* transmit events per frame                          */
    const double *tx_origin;    /* [n_tx][3] origin of each transmit wave             */
    int32_t n_lines;            /* reconstructed scanlines                            */
    const double *line_origin;  /* [n_lines][3]                                       */
    const double *line_dir;     /* [n_lines][3] unit direction                        */
    const int32_t *line_tx;     /* [n_lines] transmit event each line is formed from  */
    int32_t n_depth;            /* samples per line: r_i = depth0 + i * depth_step    */
    double depth0, depth_step;
    int32_t geometry;           /* SUPRA_GEOM_* (used by scan conversion)             */
    int32_t lines_x, lines_y;   /* line layout; lines_y = 1 for 2D                    */
    const double *tx_dir;       /* NULL, or [n_tx][3]: a nonzero row makes transmit t a plane
                                   wave of that direction passing tx_origin[t] at time 0
                                   (arrival n.(p - o_t) / c); a zero row keeps the spherical
                                   wave from tx_origin[t] (arrival |p - o_t| / c)            */
    int32_t compound;           /* 0: line l is formed from transmit line_tx[l]; 1: coherent
                                   compounding -- every line is formed from every transmit of
                                   the frame and the per-transmit images are averaged (e.g.
                                   plane waves at several angles).  Compounding plans serve
                                   delay-and-sum and the fused chain, not supra_mv or the
                                   learned apodization (SUPRA_EINVAL there).               */
} supra_scan;

/* Receive parameters (Sec. 2 item 2; dynamic aperture by F-number). */
typedef struct supra_rx {
    double c;                   /* speed of sound                                      */
    double fs;                  /* sampling rate of the channel records                */
    double fc;                  /* centre (demodulation) frequency                     */
    double fnumber;             /* aperture half width = max(z / (2 F), min_half_aperture) */
    double min_half_aperture;
    int32_t window;             /* SUPRA_WINDOW_*                                      */
    int32_t n_samples;          /* samples per channel record                          */
    double t0;                  /* time of channel sample 0 after transmit             */
} supra_rx;

/* Post-processing (Sec. 2 items 3-4). */
typedef struct supra_post {
    int32_t fir_taps;           /* odd, 1..63: IQ low-pass length                      */
    double fir_cutoff;          /* Hz (Blackman windowed sinc, unit DC gain)           */
    double dyn_range_db;        /* D: displayed dynamic range                          */
    double log_ref;             /* envelope value mapped to 0 dB (gray level 255)      */
    int32_t n_bands;            /* frequency compounding (Sec. 2 item 3): 0 or 1 = one band at
                                   fc; 2..4 = bands at fc + (k - (n_bands-1)/2) band_step, each
                                   IQ-demodulated at its centre and low-passed, envelopes averaged.
                                   Frames of plans with n_bands > 1 run the unfused chain.   */
    double band_step;           /* Hz between band centres (each centre in (0, rate/2))       */
} supra_post;

/* Cartesian output grid of scan conversion: point (ix, iy, iz) lies at
 * origin + (ix, iy, iz) * spacing; the image is stored [nz][ny][nx] (x
 * fastest) as uint8.  ny = 1 for 2D. */
typedef struct supra_grid {
    int32_t nx, ny, nz;
    double origin[3];
    double spacing[3];
} supra_grid;

typedef struct supra_plan supra_plan;

/* Sizes and algorithmic work of one frame under a plan. */
typedef struct supra_plan_info {
    int64_t n_tx, n_el, n_samples, n_lines, n_depth;
    int64_t channel_bytes;          /* n_tx * n_el * n_samples * 2: the full int16 frame             */
    int64_t aperture_element_samples; /* sum over (line, depth) of elements inside the aperture     */
    int64_t aperture_bytes;         /* 2 bytes per in-aperture element-sample                        */
    int64_t rf_bytes;               /* n_lines * n_depth * 4                                         */
    int64_t bmode_bytes;            /* n_lines * n_depth (uint8 log-compressed lines)                */
    int64_t image_bytes;            /* nx * ny * nz, or bmode_bytes without a grid                    */
    int32_t has_grid;
    int32_t depth_tile;             /* depth samples per beamforming tile                            */
} supra_plan_info;

/* Validates every parameter, copies the geometry to the device and builds the
 * resident tables (element table, per-line constants, per-tile delay bases
 * and aperture bounds, demodulation taps, log-compression constants,
 * scan-conversion inverse map).  `grid` may be NULL (no scan conversion: the
 * B-mode output is then the log-compressed lines [n_lines][n_depth]).
 * Errors: SUPRA_EINVAL (c, fs, fnumber <= 0; fc >= fs/2; n_* < 1; line_tx
 * out of range; a non-unit line direction; fir_taps even or > 63;
 * dyn_range_db <= 0; log_ref <= 0; min_half_aperture <= 0; a scanline layout that does not match
 * `geometry` when a grid is given), SUPRA_ENOMEM, SUPRA_ECUDA.  Runs on the
 * current device and is synchronous. */
SUPRA_API int supra_plan_create(const supra_probe *probe, const supra_scan *scan, const supra_rx *rx,
                      const supra_post *post, const supra_grid *grid, supra_plan **out);

/* Frees the plan's device tables (synchronous).  NULL is a no-op. */
SUPRA_API void supra_plan_destroy(supra_plan *plan);

SUPRA_API int supra_plan_get_info(const supra_plan *plan, supra_plan_info *info);

/* Receive delay-and-sum (Sec. 1 "receive beamforming"; Sec. 2 items 1-2;
 * Table 1 "Beamformer").  For line l and depth sample i the image point is
 * p = o_l + r_i d_l; element e contributes its record at
 * s = ((|p - o_t| + |p - x_e|) / c - t0) fs (t = line_tx[l]), linearly
 * interpolated, zero outside the record; apodized by the window over the
 * F-number aperture centred on (p_x, p_y) clamped to the array; the sum is
 * normalised by the sum of weights.
 *   ch: int16 [n_tx][n_el][n_samples] (device, sample-contiguous)
 *   rf: float [n_lines][n_depth]      (device)                            */
SUPRA_API int supra_beamform(const supra_plan *plan, const int16_t *ch, float *rf, void *stream);

/* IQ demodulation and envelope (Sec. 1 "envelope detection"; Sec. 2 item 3;
 * Table 1 "Envelope"): env = 2 |sum_k h_k rf(i + H - k) exp(-j 2 pi fc (i + H - k) dt)|,
 * h the plan's low-pass, H = (fir_taps - 1) / 2, dt = 2 depth_step / c,
 * zero padding at both ends of each line.
 *   rf, env: float [n_lines][n_depth] (device; may not alias)             */
SUPRA_API int supra_envelope(const supra_plan *plan, const float *rf, float *env, void *stream);

/* Log compression (Sec. 1 "log-compression"; Sec. 2 item 4; Table 1
 * "Log comp."): code = floor(255 (20 log10(env / log_ref) + D) / D + 1/2)
 * clamped to [0, 255]; env <= 0 -> 0.
 *   env: float [n_lines][n_depth], bm: uint8 [n_lines][n_depth] (device)  */
SUPRA_API int supra_logcompress(const supra_plan *plan, const float *env, uint8_t *bm, void *stream);

/* Scan conversion (Sec. 1 "scan conversion"; Sec. 2 item 5; Table 1
 * "Scan conv."): each grid point is mapped back to fractional (line,
 * depth) coordinates of the plan's layout and bilinearly (2D) or
 * trilinearly (3D) interpolated from bm, result floor(v + 1/2); points
 * outside the scanned region (more than 1e-3 index units beyond its edge)
 * are 0.  Requires a plan with a grid (else SUPRA_EINVAL).
 *   bm: uint8 [n_lines][n_depth], img: uint8 [nz][ny][nx] (device)        */
SUPRA_API int supra_scanconvert(const supra_plan *plan, const uint8_t *bm, uint8_t *img, void *stream);

/* Bytes of device workspace for the fused chain of these n frames: the
 * log-compressed lines of every frame that is scan converted (256-byte aligned
 * each; frames of frequency-compounding plans also hold their RF and
 * envelope), then the depth-segment boundary records (128 FP32 RF samples per
 * line and boundary of frames whose one-frame launches split their lines
 * along depth).  The lines are required; a workspace without room for the
 * records makes each segment beamform the 64 depths before it that its first
 * outputs filter (the same output bytes, more work).  The records follow the
 * plans' tile shapes in effect: size the workspace after setting or tuning
 * them.  0 when neither applies. */
SUPRA_API size_t supra_bmode_workspace_size(int32_t n, const supra_plan *const *plans);

/* Fused chain of one frame: beamforming, envelope and log compression in one
 * kernel that streams the frame's channel data once, then scan conversion.
 * Result equals supra_scanconvert(supra_logcompress(supra_envelope(
 * supra_beamform(ch)))) up to floating-point rounding.
 *   ch:  int16 [n_tx][n_el][n_samples] (device)
 *   out: uint8 [nz][ny][nx] with a grid, else uint8 [n_lines][n_depth]
 *   workspace: device memory of supra_bmode_workspace_size(1, &plan) bytes,
 *   256-byte aligned; at least the frame's lines (else SUPRA_EWORKSPACE); may
 *   be NULL when the plan has no grid.  Calls that share a workspace must not
 *   overlap on the device.                                                */
SUPRA_API int supra_bmode(const supra_plan *plan, const int16_t *ch, uint8_t *out, void *workspace, size_t workspace_bytes,
                void *stream);

/* Fused chain of n frames in one launch per stage (n >= 1).  Frames may use
 * different plans (uneven 2D/3D sizes); consecutive frames that share a plan
 * are beamformed together so their delays and weights are computed once.
 * plans, ch, out: host arrays of n entries (device data pointers as for
 * supra_bmode).  workspace: supra_bmode_workspace_size(n, plans) bytes.   */
SUPRA_API int supra_bmode_batched(int32_t n, const supra_plan *const *plans, const int16_t *const *ch, uint8_t *const *out,
                        void *workspace, size_t workspace_bytes, void *stream);

/* Exact minimum-variance (Capon) beamformer.  The paper has no MV node; it
 * labels the training data of the learned apodization and serves as its
 * fallback and judge.  Per pixel: the delayed, interpolated samples x of the
 * elements inside the F-number aperture (the delays and aperture of
 * supra_beamform, no apodization), M of them in element order; subapertures
 * x_l = x[l : l + L], L = min(subaperture, M), K = M - L + 1;
 * R = (1/K) sum_l x_l x_l^T + loading * (trace(R) / L) * I (loading relative
 * to the mean eigenvalue); w = R^{-1} 1 / (1^T R^{-1} 1);
 * rf = w^T (1/K) sum_l x_l.  M < 2: the delay-and-sum value.  Solved in FP32
 * when subaperture / loading <= 1e4 (the loading bounds the condition number
 * by 1 + L/loading), else in FP64.
 *   subaperture: 1..32; loading > 0, finite (0.01 is the usual choice)
 *   ch: int16 [n_tx][n_el][n_samples], rf: float [n_lines][n_depth] (device)
 * Errors: SUPRA_EINVAL (arguments; an aperture that can hold more than 256
 * elements). */
SUPRA_API int supra_mv(const supra_plan *plan, int32_t subaperture, float loading, const int16_t *ch, float *rf,
                       void *stream);

/* ------------------------------------------------------------------------
 * Learned apodization.  The paper has no learned beamformer; this per-pixel
 * network stands in for supra_mv at delay-and-sum cost.  For each pixel, x =
 * the delayed samples of all n_el <= 128 elements (delays and F-number
 * aperture of supra_beamform, 0 outside the aperture), xh = x / ||x||:
 *   h1 = relu(W1 xh + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3,
 *   w = softmax of z over the aperture, y = sum_e w_e x_e.
 * params: float [SUPRA_APOD_PARAMS] (device) = W1 [64][128], b1 [64],
 * W2 [64][64], b2 [64], W3 [128][64], b3 [128], row-major [out][in].  The
 * products run on BF16 tensor cores with FP32 accumulation (weights and
 * activations rounded to BF16); softmax and output in FP32.
 * Training data: a feature row per pixel = BF16 [128] (xh), mask = uint32 [4]
 * (bit e of word e / 32 = element e in the aperture), norm = ||x|| (float),
 * label = the target beamformed value (e.g. supra_mv); the loss is the mean
 * over pixels with ||x|| > 0 of (sum_e w_e xh_e - label / ||x||)^2.
 * Rows of pixel k: base + k * stride (stride >= 1 rows).  feat and mask must
 * be 16-byte aligned.  All pointers are device pointers.
 * ------------------------------------------------------------------------ */
#define SUPRA_APOD_PARAMS 20736
#define SUPRA_APOD_INPUTS 128

/* Feature rows of every pixel of a frame, pixel index line * n_depth + i:
 * feat bf16 [n_lines * n_depth][128], mask uint32 [..][4], norm float [..].
 * Errors: SUPRA_EINVAL (n_el > 128, misaligned pointers). */
SUPRA_API int supra_apod_features(const supra_plan *plan, const int16_t *ch, uint16_t *feat, uint32_t *mask,
                                  float *norm, void *stream);

/* Network on n feature rows: y[k * stride] = ||x|| * sum_e w_e xh_e. */
SUPRA_API int supra_apod_forward(const float *params, int64_t n, int64_t stride, const uint16_t *feat,
                                 const uint32_t *mask, const float *norm, float *y, void *stream);

/* Bytes of workspace supra_apod_grad needs on the current device (per-CTA
 * partial gradients). */
SUPRA_API size_t supra_apod_workspace_size(void);

/* Loss and its gradient over n rows: grad float [SUPRA_APOD_PARAMS], loss
 * float [1] (may be NULL).  Deterministic for a given device.
 * Errors: SUPRA_EINVAL, SUPRA_EWORKSPACE (workspace too small). */
SUPRA_API int supra_apod_grad(const float *params, int64_t n, int64_t stride, const uint16_t *feat,
                              const uint32_t *mask, const float *norm, const float *label, float *grad, float *loss,
                              void *workspace, size_t workspace_bytes, void *stream);

/* One Adam step in place (step counts from 1; bias-corrected moments m, v,
 * each float [SUPRA_APOD_PARAMS]). */
SUPRA_API int supra_apod_adam(float *params, float *m, float *v, const float *grad, int32_t step, float lr,
                              float beta1, float beta2, float eps, void *stream);

/* One training step: supra_apod_grad on the given rows (grad and loss written
 * as it writes them), then supra_apod_adam with that gradient, the gradient
 * reduction and the update fused into one kernel.  Arguments, ownership and
 * errors as the two calls (step counts from 1). */
SUPRA_API int supra_apod_step(float *params, float *m, float *v, int32_t step, float lr, float beta1, float beta2,
                              float eps, int64_t n, int64_t stride, const uint16_t *feat, const uint32_t *mask,
                              const float *norm, const float *label, float *grad, float *loss, void *workspace,
                              size_t workspace_bytes, void *stream);

/* One epoch of training: n_batches minibatch steps (as supra_apod_step),
 * issued by the library (no per-step round trip through the caller).  The
 * rows are cut into chunks of `chunk` consecutive rows (1, or 128 = one tile
 * of the gradient kernel; the last chunk may be partial) and minibatch b takes
 * the chunks order[b], order[b] + n_batches, order[b] + 2 n_batches, ...
 * (interleaved minibatches; order: host array, a permutation of 0 ..
 * n_batches - 1); it is Adam step step0 + b + 1, losses[b] (device float
 * [n_batches]) receives its mean loss, grad the last step's gradient.  With
 * chunk = 1 every step equals supra_apod_step(rows order[b], stride
 * n_batches); with 128 each tile reads consecutive rows (one contiguous
 * block of feature rows per tile instead of rows n_batches apart).
 * Errors: SUPRA_EINVAL (chunk not 1 or 128, order entries out of range,
 * fewer chunks than minibatches), else as supra_apod_step, returned at the
 * first failing step. */
SUPRA_API int supra_apod_epoch(float *params, float *m, float *v, int32_t step0, float lr, float beta1, float beta2,
                               float eps, int64_t n_rows, int32_t n_batches, int32_t chunk, const int32_t *order,
                               const uint16_t *feat, const uint32_t *mask, const float *norm, const float *label,
                               float *grad, float *losses, void *workspace, size_t workspace_bytes, void *stream);

/* Learned-apodization beamformer: rf float [n_lines][n_depth] from int16
 * channels [n_tx][n_el][n_samples], delays, interpolation and aperture as in
 * supra_beamform, weights from the network (one fused kernel).
 * Errors: SUPRA_EINVAL (n_el > 128). */
SUPRA_API int supra_apod_mlp(const supra_plan *plan, const float *params, const int16_t *ch, float *rf, void *stream);

/* ------------------------------------------------------------------------
 * Headless volume rendering of a scan-converted volume (the paper shows
 * rendered 3D output, Fig. 4b; no graphics API: the image is a device
 * buffer).  Orthographic ray march: pixel (px, py) of a width x height image
 * casts the ray from centre + (px - (width-1)/2) right + (py - (height-1)/2)
 * down along the unit direction dir, sampled at t0 + k dt, k < n_steps
 * (metres).  Samples are trilinear in the uint8 volume [nz][ny][nx] laid on
 * `grid`, 0 outside.  SUPRA_RENDER_MIP: image = maximum sample (0..255).
 * SUPRA_RENDER_EA: front-to-back emission-absorption, a = clamp((v - lo) /
 * (hi - lo), 0, 1) alpha, c = v / 255, C = sum T a c, T *= 1 - a (0..1).
 * vol, image: device pointers; image float [height][width].
 * Errors: SUPRA_EINVAL (sizes, a zero ray direction, hi <= lo).
 * ------------------------------------------------------------------------ */
enum { SUPRA_RENDER_MIP = 0, SUPRA_RENDER_EA = 1 };

typedef struct {
    double centre[3], right[3], down[3], dir[3];
    double t0, dt;
    int32_t n_steps, width, height, mode;
    double lo, hi, alpha;
} supra_camera;

SUPRA_API int supra_render(const supra_grid *grid, const uint8_t *vol, const supra_camera *cam, float *image,
                           void *stream);

/* ------------------------------------------------------------------------
 * Tuning (no counterpart in the paper, whose nodes have fixed launch
 * shapes).  A plan carries the tile shape its frames are beamformed with:
 *   frames_per_group    1, 2, 4, 8 or 16: frames of one plan that are adjacent
 *                       in a batch share a DAS tile (frames x 256 depths x 1
 *                       line) -- larger tiles share the delay and weight
 *                       arithmetic across frames, smaller ones expose more
 *                       tiles to the SMs;
 *   elements_per_stage, stages
 *                       16-frame groups: element windows per staging-ring
 *                       stage and ring depth, 3 x 3 (default) or 2 x 4;
 *   depth_segments      0 = automatic (lines split along depth so that a
 *                       launch with few lines fills one wave), k >= 1: k
 *                       segments per line (1 = whole lines), at most 64;
 *                       16-frame groups always keep whole lines;
 *   ctas_per_sm         one-frame launches: 0 = automatic, 2 or 3 resident
 *                       CTAs per SM (registers sized for that many).
 * A batched launch that mixes plans takes depth_segments and ctas_per_sm from
 * its first frame's plan.  Set before the plan is shared across threads.
 * ------------------------------------------------------------------------ */
typedef struct supra_tile_shape {
    int32_t frames_per_group;
    int32_t elements_per_stage;
    int32_t stages;
    int32_t depth_segments;
    int32_t ctas_per_sm;
} supra_tile_shape;

/* SUPRA_EINVAL for a value outside the lists above. */
SUPRA_API int supra_plan_set_tile_shape(supra_plan *plan, const supra_tile_shape *shape);
SUPRA_API int supra_plan_get_tile_shape(const supra_plan *plan, supra_tile_shape *shape);
/* frames_per_group alone (the other settings unchanged). */
SUPRA_API int supra_plan_set_max_group(supra_plan *plan, int32_t max_group);   /* 1, 2, 4, 8 or 16 */
SUPRA_API int32_t supra_plan_get_max_group(const supra_plan *plan);

/* Autotuner: times supra_bmode_batched of n frames of `plan` (device
 * pointers as for supra_bmode_batched; outputs are overwritten) with CUDA
 * events on `stream` (reps timed calls after one warm-up each) for the shape
 * in effect and then for each frames-per-group class crossed with the
 * settings its launches use (stage shapes of 16-frame groups; depth segments
 * 0 to 6 and 8 of the others; CTAs per SM 0, 2, 3 of one-frame launches),
 * keeps the fastest shape in the plan and returns it with its time per call
 * and the time of the shape in effect before (start_ms; may be NULL).  The
 * outputs do not depend on the shape.  Trials that need more workspace than
 * the one given (shapes with more depth segments) run in a temporary one it
 * allocates and frees.  Synchronizes the stream; on an error the plan keeps
 * its shape. */
SUPRA_API int supra_autotune_tile_shape(supra_plan *plan, int32_t n, const int16_t *const *ch, uint8_t *const *out,
                                        void *workspace, size_t workspace_bytes, int32_t reps, void *stream,
                                        supra_tile_shape *best, float *best_ms, float *start_ms);
/* The same search, returning only the frames-per-group class it picked. */
SUPRA_API int supra_autotune_bmode(supra_plan *plan, int32_t n, const int16_t *const *ch, uint8_t *const *out,
                                   void *workspace, size_t workspace_bytes, int32_t reps, void *stream,
                                   int32_t *best_group, float *best_ms);

/* ------------------------------------------------------------------------
 * Real-time request loop.  The paper's runtime streams frames through its
 * processing graph (Sec. 2); this server runs many acquisitions at once on one
 * GPU: a device arena of memory_bytes is allocated at creation and every
 * request's footprint (ingested channels, output, scratch) is reserved from
 * it in arrival order; admitted requests of one kind form the next batch
 * (B-mode frames of any plans in one uneven supra_bmode_batched call, frames
 * of one plan side by side); batches run round-robin on n_streams streams;
 * with use_graphs, a batch whose (stream, kind, plan sequence) bucket has
 * been seen before replays that bucket's CUDA graph (updated in place for the
 * new buffers), a first-seen bucket launches directly.  Results
 * are B-mode images (the plan's grid, else its log-compressed lines) by the
 * request's beamformer: fused delay-and-sum, minimum variance, or learned
 * apodization, each followed by envelope, log compression and scan
 * conversion.  Times are seconds on the server's clock.
 * ------------------------------------------------------------------------ */
typedef struct supra_server supra_server;

enum { SUPRA_KIND_DAS = 0, SUPRA_KIND_MV = 1, SUPRA_KIND_APOD = 2 };

typedef struct {
    size_t memory_bytes;  /* device arena for ingested channels, outputs and scratch */
    int32_t n_streams;    /* 1..64 */
    int32_t max_batch;    /* requests per batch (B-mode: frames per supra_bmode_batched call) */
    int32_t use_graphs;   /* capture batches into CUDA graphs */
} supra_server_config;

typedef struct {
    int32_t kind;                 /* SUPRA_KIND_* */
    const supra_plan *plan;       /* resident plan, alive until the request completes */
    const int16_t *ch;            /* device channels read in place, or NULL */
    const int16_t *ch_host;       /* host channels (pinned for overlap) copied into the arena, or NULL */
    uint8_t *out_host;            /* host destination of the result, or NULL: result stays in the arena */
    const float *apod_params;     /* SUPRA_KIND_APOD: device float [SUPRA_APOD_PARAMS] */
    int32_t mv_subaperture;       /* SUPRA_KIND_MV: 1..32 */
    float mv_loading;             /* SUPRA_KIND_MV: > 0 */
    int64_t tag;                  /* returned in the completion */
} supra_request;

typedef struct {
    int64_t ticket, tag;
    int32_t status;               /* SUPRA_OK or an error code */
    int32_t batch_size;           /* requests in the batch it ran in */
    const uint8_t *out;           /* device result when out_host was NULL (valid until supra_server_release) */
    int64_t out_bytes;
    double t_submit, t_admit, t_done;   /* arrival, memory admission, completion on the device */
} supra_completion;

typedef struct {
    int64_t submitted, completed, batches, graph_launches, graph_instantiations, graph_updates;
    int64_t memory_used, memory_peak;
    int32_t pending, inflight;
} supra_server_stats;

/* Errors: SUPRA_EINVAL, SUPRA_ENOMEM (arena), SUPRA_ECUDA. */
SUPRA_API int supra_server_create(const supra_server_config *cfg, supra_server **out);
/* Queues one request (thread-safe).  SUPRA_EINVAL: bad request, or one that
 * cannot fit the arena even alone. */
SUPRA_API int supra_server_submit(supra_server *s, const supra_request *req, int64_t *ticket);
/* Open-loop arrivals: request i is submitted at t_arrival[i] seconds
 * (non-decreasing) after this call by a feeder thread; latencies count from
 * the scheduled arrival.  tickets[i] (may be NULL) receives its ticket. */
SUPRA_API int supra_server_submit_trace(supra_server *s, int32_t n, const supra_request *reqs,
                                        const double *t_arrival, int64_t *tickets);
/* Up to max completed requests, oldest first (non-blocking). */
SUPRA_API int supra_server_poll(supra_server *s, supra_completion *out, int32_t max, int32_t *n);
/* Blocks until n_submitted requests have been submitted and none is pending or
 * running; SUPRA_ETIMEOUT after timeout_s seconds. */
SUPRA_API int supra_server_wait(supra_server *s, int64_t n_submitted, double timeout_s);
/* Frees the arena memory of a result kept on the device. */
SUPRA_API int supra_server_release(supra_server *s, int64_t ticket);
SUPRA_API int supra_server_get_stats(supra_server *s, supra_server_stats *stats);
SUPRA_API double supra_server_now(const supra_server *s);
/* Finishes all submitted work, then frees everything. */
SUPRA_API void supra_server_destroy(supra_server *s);

/* supra_bmode for callers that may not allocate device memory.  The paper has
 * no counterpart: it exists because some callers cannot provide the device
 * workspace supra_bmode needs -- e.g. a real-time acquisition loop that must
 * not call cudaMalloc after start-up (it can synchronize the device and has no
 * latency bound), or a host whose device memory belongs to another
 * framework's pool.  It runs the same kernels as supra_bmode, taking the
 * scratch for the frame's log-compressed lines from a fixed 8 MiB array in the
 * library's device memory, and allocates nothing.
 *   - Frames whose required workspace exceeds 8 MiB (8388608 bytes) are
 *     rejected with SUPRA_EINVAL before anything is launched.  That is
 *     n_lines * n_depth bytes for one-band plans with a grid; plans with
 *     frequency compounding (n_bands > 1) also need two FP32 RF-sized buffers
 *     (9 bytes per line sample), so their frames may be 1/9 as large.  The
 *     depth-segment boundary records use the rest of the array when they fit.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and keeps it for that device's context; make that
 *     first call before any stream capture.  After a device reset the next
 *     call looks it up again (it also counts as a first call).
 *   - Every call on a device uses the same array and leaves its contents
 *     behind; calls whose work overlaps on the GPU (different streams, host
 *     threads) race on it and must be ordered by the caller.  No part of the
 *     array needs to start at zero: each call overwrites what it reads.
 *   Arguments as for supra_bmode without the workspace. */
SUPRA_API int supra_bmode_noalloc(const supra_plan *plan, const int16_t *ch, uint8_t *out, void *stream);

/* Reads (and, if clear != 0, resets) the device status word of the current
 * device: 0 = no device-side failure since the last clear, else the
 * negative SUPRA_E* code of the first failure.  Synchronizes the device. */
SUPRA_API int supra_device_status(int32_t clear);

/* Self-test of the bounded device waits that every kernel's mbarrier waits use.
 * Launches one CTA of 96 threads on the current device (default stream) whose
 * mbarrier never completes (nothing arrives on it):
 *   - thread 0 waits with a budget of budget_cycles SM clock cycles;
 *   - thread 32 waits as the beamforming kernel's stage consumers do, giving up
 *     when the CTA's abort word is raised, which thread 64 does after
 *     budget_cycles cycles of its own (bounded spin on clock64).
 * Both waits give up, set the device status word to SUPRA_ETIMEOUT and return;
 * the context stays usable (read and clear the word with supra_device_status).
 * budget_cycles: 1 << 10 .. 1 << 31.  out_host (host, may be NULL): int32[2],
 * element k = 1 where wait k reported the timeout.  Returns SUPRA_OK,
 * SUPRA_EINVAL (budget out of range, before any CUDA call) or SUPRA_ECUDA.
 * Synchronizes the device. */
SUPRA_API int supra_selftest_bounded_wait(int64_t budget_cycles, int32_t *out_host);

/* Static description of a return code. */
SUPRA_API const char *supra_strerror(int code);

/* Library version string. */
SUPRA_API const char *supra_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SUPRA_H */
