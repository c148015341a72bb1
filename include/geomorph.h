/*
 * geomorph -- geodesic 3x3 chains on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library libgeomorph.so. Every function is extern "C", takes
 * plain pointers and sizes, and returns a geo_status (0 = success). Nothing
 * is thrown across the boundary.
 *
 * The operations follow Zlaus & Mongus, "Efficient method for parallel
 * computation of geodesic transformation on CPU" (IEEE TPDS 2019):
 *
 *   image model        Section 2: f : P -> R, P = {0..X-1} x {0..Y-1},
 *                      X = width, Y = height, stored row-major.
 *   neighbourhood      Section 2, Eq. 1-2: the 3x3 square w_1(p) clipped to
 *                      the image (pixels outside P are ignored, never padded).
 *                      conn = 8 selects it; conn = 4 selects the cross
 *                      {centre, left, right, up, down}, also clipped, which
 *                      the paper does not use (an extension of this library).
 *   elementary step    Section 2, Eq. 3: erosion  f' = max(eps_1(f), m),
 *                      dilation f' = min(delta_1(f), m). Every step is
 *                      computed from the whole previous image.
 *   chain              Section 2, Eq. 4: `steps` nested elementary steps.
 *   reconstruction     Section 2, Eq. 5: the limit of the chain, reached
 *                      when a step changes no pixel (Section 3.7, Algorithm 5).
 *   square window      Section 2, Eq. 1-2 with half size s: the clipped
 *                      (2s+1)^2 window, computed as s unmasked 3x3 steps
 *                      (the decomposition of Section 3.1).
 *
 * Common conventions
 *   - Pointers named marker, mask, in, out, grad_* are DEVICE pointers owned
 *     by the caller. The library reads marker/mask/in and writes out; it
 *     never frees or keeps them after the call's GPU work completes.
 *   - Element type: GEO_U8 (uint8_t), GEO_F32 (float), GEO_F64 (double).
 *     NaN and negative zero are outside the contract.
 *   - `pitch` is the row stride in ELEMENTS (pitch >= width), shared by all
 *     image arguments of a call. Pixel (y, x) is at ptr[y * pitch + x].
 *   - `out` may alias `marker` (in-place); `out` must not overlap `mask`.
 *   - height == 0 or width == 0 is a no-op returning GEO_OK.
 *   - Every call is asynchronous on `stream` (a cudaStream_t, may be NULL for
 *     the legacy default stream). Internal scratch memory is allocated
 *     stream-ordered (cudaMallocAsync from a library-owned pool) and released
 *     stream-ordered before the call returns.
 *   - Errors a call can detect on the host (bad arguments, launch failure)
 *     are returned directly. Errors detected on the device (a bounded wait
 *     that expired, a reconstruction that did not converge) are recorded in
 *     a per-device status word: read it with geo_device_status(). The word
 *     keeps the first error until it is read; while it holds one, kernels
 *     that meet at a grid barrier stop at their next barrier (their output
 *     is then incomplete), so read it before trusting later results.
 *   - One library instance serves every device; calls use the current device.
 */
#ifndef GEOMORPH_H
#define GEOMORPH_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GEO_API __attribute__((visibility("default")))
#else
#define GEO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { GEO_U8 = 0, GEO_F32 = 1, GEO_F64 = 2 } geo_dtype;

typedef enum {
    GEO_OK = 0,
    GEO_ERR_ARG = -1,            /* invalid argument (pointer, size, pitch, conn, steps, aliasing) */
    GEO_ERR_DTYPE = -2,          /* unsupported element type for this operation */
    GEO_ERR_ALIGN = -3,          /* pointer not aligned to its element size */
    GEO_ERR_CUDA = -4,           /* a CUDA runtime call failed (launch, allocation, ...) */
    GEO_ERR_TIMEOUT = -5,        /* device: a bounded inter-block wait expired */
    GEO_ERR_NOT_CONVERGED = -6,  /* device: reconstruction hit max_steps while still changing */
    GEO_ERR_WORKSPACE = -7       /* caller-provided workspace too small */
} geo_status;

/* Human-readable name of a geo_status value (static string). */
GEO_API const char *geo_status_string(int status);

/*
 * Reads and clears the device status words of the current device after
 * synchronising `stream`: the library's word and the word of
 * geo_dilate_chain_noalloc. *status receives GEO_OK or the first device-side
 * error (GEO_ERR_TIMEOUT, GEO_ERR_NOT_CONVERGED) recorded since the last
 * read (the library's word first). Allocates nothing. Returns GEO_ERR_CUDA
 * if the synchronisation or a copy failed.
 */
GEO_API int geo_device_status(void *stream, int *status);

/*
 * Geodesic dilation of size `steps` (Eq. 4 with the dilation step of Eq. 3's
 * dual): out = delta^mask_steps(marker), each step f' = min(delta_1(f), mask).
 * steps >= 0 (0 copies marker to out). conn is 4 or 8. mask must not be NULL.
 */
GEO_API int geo_dilate_chain(geo_dtype dtype, const void *marker, const void *mask, void *out,
                     int64_t height, int64_t width, int64_t pitch, int conn,
                     int64_t steps, void *stream);

/* Geodesic erosion of size `steps` (Eq. 3-4): each step f' = max(eps_1(f), mask). */
GEO_API int geo_erode_chain(geo_dtype dtype, const void *marker, const void *mask, void *out,
                    int64_t height, int64_t width, int64_t pitch, int conn,
                    int64_t steps, void *stream);

/*
 * Reconstruction (Eq. 5): op = 0 dilation by reconstruction delta^mask_rec,
 * op = 1 erosion by reconstruction eps^mask_rec. Steps are applied until a
 * step changes no pixel. The device loop runs whole passes of several steps,
 * so it may apply a few steps past the fixed point; those change nothing.
 * max_steps caps the number of steps applied, counted in whole passes
 * (<= 0: height * width + 1 + 1024, which covers the changing steps of any
 * input, at most height * width + 1, plus the pass that detects the fixed
 * point); a pass that reaches the cap and still changed a pixel records
 * GEO_ERR_NOT_CONVERGED in the device status word (the image reached so far
 * is left in out).
 * steps_out: optional DEVICE int64_t*; receives the number of steps applied
 * (an upper bound on the changing steps, rounded up to whole passes).
 */
GEO_API int geo_reconstruct(geo_dtype dtype, const void *marker, const void *mask, void *out,
                    int64_t height, int64_t width, int64_t pitch, int conn, int op,
                    int64_t max_steps, int64_t *steps_out, void *stream);

/*
 * Dilation (Eq. 2) / erosion (Eq. 1) by the clipped square window of half
 * size half_size >= 0, i.e. a (2s+1) x (2s+1) window, computed as half_size
 * unmasked 8-connected 3x3 steps. out may alias in.
 */
GEO_API int morph_window_dilate(geo_dtype dtype, const void *in, void *out, int64_t height,
                        int64_t width, int64_t pitch, int64_t half_size, void *stream);
GEO_API int morph_window_erode(geo_dtype dtype, const void *in, void *out, int64_t height,
                       int64_t width, int64_t pitch, int64_t half_size, void *stream);

/*
 * Geodesic operators of Section 2 built on reconstruction. f is the input
 * image (also the mask of the reconstruction), out the result; out must not
 * overlap f. Values that the operators produce by subtraction are computed in
 * the element type (uint8 saturates at 0; float32 rounds to float32).
 * geo_hmax      HMAX_h(f) = delta_rec^f(f - h)            (Eq. 6), h >= 0
 *               (uint8: h rounded down, at most 255)
 * geo_dome      DOME_h(f) = f - HMAX_h(f)                 (Eq. 7)
 * geo_hfill     HFILL(f) = eps_rec^f(m), m = f on the image border and
 *               max f inside                              (Eq. 8-9)
 * geo_raobj     RAOBJ(f) = f - delta_rec^f(m), m = f on the border and
 *               min f inside                              (Eq. 10-11)
 * geo_open_rec  gamma_rec^s(f) = delta_rec^f(eps_s(f)), eps_s the clipped
 *               (2s+1)^2 square erosion                   (Eq. 12)
 * conn (4 or 8) is the connectivity of the reconstruction. Asynchronous on
 * stream; device-side non-convergence is reported by geo_device_status.
 */
GEO_API int geo_hmax(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch,
             int conn, double h, void *stream);
GEO_API int geo_dome(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch,
             int conn, double h, void *stream);
GEO_API int geo_hfill(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch,
              int conn, void *stream);
GEO_API int geo_raobj(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch,
              int conn, void *stream);
GEO_API int geo_open_rec(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width,
                 int64_t pitch, int conn, int64_t half_size, void *stream);

/*
 * Quasi-distance transform (Section 2, Eq. 13-15; Section 3.8, Algorithm 6).
 *
 * Part 1: f is eroded S times with eps_1 (the 3x3 square for conn = 8, the
 * cross for conn = 4; clipped to the image), S = max(H, W) - 1 (conn 8) or
 * H + W - 2 (conn 4), after which the erosion is constant. After erosion j
 * the residual eps_{j-1}(f) - eps_j(f) of each pixel replaces r and j
 * replaces d where it is strictly larger than the r kept so far (r and d
 * start at 0; equal residuals keep the earlier j).
 * Part 2: d_l1 = the limit of eta (Eq. 14) applied to d, eta(g) =
 * eps_1(g) + 1 where g - eps_1(g) > 1 and g elsewhere.
 *
 * dtype     GEO_U8 only (else GEO_ERR_DTYPE).
 * f         device, H rows of `pitch` uint8 elements; read only.
 * r         device uint8, same layout as f: the largest residual.
 * d         device int32, H rows of `pitch` int32 elements: the first
 *           erosion index attaining r (0 where no erosion lowers the pixel).
 * d_l1      device int32 like d, or NULL to skip part 2; may equal d (then
 *           d is overwritten by the limit).
 * r, d and d_l1 (unless equal to d) must not overlap f or one another.
 * Errors: GEO_ERR_ARG for negative sizes, pitch < width, conn not 4 or 8,
 * NULL f, r or d, overlapping buffers, or S > 32766; GEO_ERR_ALIGN when d or
 * d_l1 is not 4-byte aligned. Asynchronous on stream; a device-side wait
 * timeout or non-convergence is reported by geo_device_status. The library
 * allocates its scratch from its stream-ordered pool.
 */
GEO_API int geo_qdt(geo_dtype dtype, const void *f, void *r, int32_t *d, int32_t *d_l1, int64_t height,
                    int64_t width, int64_t pitch, int conn, void *stream);

/*
 * Openings, closings, granulometry and alternating sequential filters
 * (Section 2, Eq. 16-20), all with the 3x3 square (the paper's w_1) clipped
 * to the image, eps_s / delta_s being s chained elementary steps:
 *
 * geo_opening       gamma_s(f) = delta_s(eps_s(f))                  (Eq. 16)
 * geo_closing       phi_s(f)   = eps_s(delta_s(f))                  (Eq. 19)
 * geo_asf           ASF_s(f) = phi_s(gamma_s(... phi_1(gamma_1(f))))  (Eq. 20)
 * geo_granulometry  G_k = sum over the image of gamma_k(f) for k = 0..smax
 *                   (Eq. 17) and PS_k = G_k - G_{k+1} for k = 0..smax-1
 *                   (Eq. 18)
 *
 * f, out: device images of `dtype`, H rows of `pitch` elements; out may
 * equal f (in place) but must not otherwise overlap it. half_size / s >= 0
 * (0: out = f). G: device double[smax + 1]; PS: device double[smax] or NULL;
 * both 8-byte aligned. G sums in double with a fixed order: exact for
 * uint8, deterministic for floats. Errors: GEO_ERR_DTYPE, GEO_ERR_ARG
 * (negative sizes, pitch < width, NULL pointers, overlap), GEO_ERR_ALIGN.
 * Asynchronous on stream; scratch comes from the library's pool.
 */
GEO_API int geo_opening(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch,
                        int64_t half_size, void *stream);
GEO_API int geo_closing(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch,
                        int64_t half_size, void *stream);
GEO_API int geo_asf(geo_dtype dtype, const void *f, void *out, int64_t height, int64_t width, int64_t pitch,
                    int64_t s, void *stream);
GEO_API int geo_granulometry(geo_dtype dtype, const void *f, int64_t height, int64_t width, int64_t pitch,
                             int64_t smax, double *G, double *PS, void *stream);

/*
 * Batched execution: many independent items in one persistent launch.
 * The paper has no batched form; item i computes exactly what the matching
 * single-item entry point computes on its own images.
 */
typedef struct {
    int op;              /* 0 dilation chain, 1 erosion chain (Eq. 3-4),
                            2 dilation by reconstruction, 3 erosion by reconstruction (Eq. 5),
                            4 window dilation, 5 window erosion (Eq. 1-2) */
    geo_dtype dtype;
    int conn;            /* 4 or 8; windows are always the 8-connected square */
    int64_t height, width, pitch;  /* pitch in elements, >= width */
    int64_t steps;       /* chain: steps (>= 0); window: half size s (>= 0);
                            reconstruction: max_steps (<= 0: default as geo_reconstruct) */
    const void *marker;  /* device input (the image, for windows) */
    const void *mask;    /* device mask (ignored for windows) */
    void *out;           /* device output; may alias marker, must not overlap mask */
} geo_item;

/*
 * Bytes of device workspace geo_batch needs for these items (descriptor
 * table, per-item state, the tile work-queue, one scratch image per item);
 * 0 if an item is invalid.
 */
GEO_API size_t geo_batch_workspace_size(const geo_item *items, int n);

/*
 * geo_batch = geo_batch_prepare + geo_batch_launch.
 * geo_batch_prepare uploads the items' descriptors (tile geometry, K per
 *   item) from host memory into the workspace; stream-ordered. It also sets
 *   up the library's state on the current device (allocated on first use),
 *   so that the launch that follows allocates nothing.
 * geo_batch_launch resets the queue and runs every item to completion in one
 *   persistent cooperative kernel; it copies nothing from the host, so a
 *   prepared workspace can be launched repeatedly (and captured in a CUDA
 *   graph) as long as the items' pointers and sizes are unchanged.
 * status_out: optional DEVICE int[n]; item i gets GEO_OK,
 *   GEO_ERR_NOT_CONVERGED (reconstruction cap reached) or GEO_ERR_TIMEOUT
 *   (the launch ended before the item completed).
 * Items are scheduled largest first; a tile of an item waits only for its
 * own item's previous pass. Workspace contents must not be modified between
 * prepare and launch.
 */
GEO_API int geo_batch_prepare(const geo_item *items, int n, void *workspace, size_t ws_bytes, void *stream);
GEO_API int geo_batch_launch(const geo_item *items, int n, void *workspace, int *status_out, void *stream);
GEO_API int geo_batch(const geo_item *items, int n, void *workspace, size_t ws_bytes, int *status_out,
              void *stream);

/*
 * Autotuning of the batch's tiles (not in the paper). The batch planner gives
 * each item the pass length K that minimises tile-steps plus a per-pass
 * charge (the hand-over between passes and the queue), in units of one
 * region-step; the charge is the tuned policy. geo_batch_autotune prepares
 * and launches these items with each candidate charge (2.5, 5, 10, 20, 40,
 * 80), times two launches after a warm-up with CUDA events on `stream`,
 * keeps the fastest under which every item completed (status_out, if given,
 * is checked), stores it in the library's tune table (written to cache_path
 * if not NULL, with the rest of the table) for every later
 * geo_batch_prepare, and leaves the workspace prepared with it. Synchronous;
 * the items' outputs are overwritten. Untuned, the charge is 10.
 */
GEO_API int geo_batch_autotune(const geo_item *items, int n, void *workspace, size_t ws_bytes, int *status_out,
                               void *stream, const char *cache_path);

/*
 * Autotuning of the register kernel's tiles, persisted. The paper has no
 * counterpart (its CPU pipeline has no tile size). What is searched: the pass
 * length K (which fixes the tile interior) and the kernel's shape variant
 * (band height and warps per block, hence the region and the block size):
 * for uint8, variant 0 = 128x128 pixels / 512 threads, 1 = 128x64 / 256,
 * 2 = 128x96 / 384; for float32, 0 = 128x128 / 512, 1 = 128x64 / 256 (8-row
 * bands), 2 = 128x64 / 512 (4-row bands); float64 has variant 0 only.
 * geo_autotune times every valid (variant, K) for each item (a geo_item as
 *   above; the call runs the item's operation on its own buffers several
 *   times, so out is overwritten), keeps the fastest per (dtype, op, conn,
 *   height, width, chain-length class) and per (dtype, op, conn, size class
 *   of height, of width, chain-length class) in the library's tune table
 *   (size classes are half octaves, floor(2 log2 n); a class keeps the
 *   choice of the largest item tuned in it) and, if cache_path is not NULL,
 *   writes the whole table there. Each entry also keeps the fastest K of
 *   variant 0, which the batch kernel (one block size for every item) uses.
 *   Synchronous. GEOMORPH_K and GEOMORPH_VARIANT must not be set
 *   (GEO_ERR_ARG).
 * geo_tune_load reads such a file into the tune table (entries from any
 *   device). The environment variable GEOMORPH_TUNE_CACHE names a file that
 *   is loaded on first use, keeping only entries tuned on the same device
 *   model.
 * geo_tune_reset empties the tune table (the planners' cost models decide
 *   again; a GEOMORPH_TUNE_CACHE file is not read a second time).
 * geo_tune_save writes the tune table to a file (the format geo_tune_load
 *   reads).
 * Lookups take the exact (height, width) entry, else its size class.
 * geo_tune_lookup returns the tuned K of variant 0 for that key, or 0. Chain
 *   lengths of 64 and more share one class; reconstruction ignores steps.
 * geo_plan_info reports the K and tile interior (TH x TW) the single-image
 *   entry points use for these arguments (op as in geo_item);
 *   geo_plan_shape also the shape variant and the threads per block.
 */
GEO_API int geo_autotune(const geo_item *items, int n, const char *cache_path);
GEO_API int geo_tune_load(const char *cache_path);
GEO_API int geo_tune_reset(void);
GEO_API int geo_tune_save(const char *cache_path);
GEO_API int geo_tune_lookup(int dtype, int op, int conn, int64_t height, int64_t width, int64_t steps);
GEO_API int geo_plan_info(geo_dtype dtype, int op, int conn, int64_t height, int64_t width, int64_t steps,
                  int *K, int *TH, int *TW);
GEO_API int geo_plan_shape(geo_dtype dtype, int op, int conn, int64_t height, int64_t width, int64_t steps,
                           int *K, int *TH, int *TW, int *variant, int *threads);

/*
 * Reverse mode of the masked chain (Eq. 4) for GEO_F32 / GEO_F64; the paper
 * has no backward pass, these are this library's rules. A step computes
 * f_t(p) = clamp(ext_{q in N(p)} f_{t-1}(q), m(p)) (ext = max and clamp =
 * min for dilation, op = 0; the reverse for erosion, op = 1). Its upstream
 * gradient g_t(p) goes to the mask at p when the mask is strictly beyond the
 * neighbourhood extreme, otherwise to f_{t-1}(p + d_k) with k = (dy+1)*3 +
 * (dx+1) the lowest neighbour index attaining the extreme. Gradients are
 * summed as a gather over k = 0..8 in increasing order, in the element type;
 * grad_mask accumulates over steps N, N-1, ..., 1. Results are deterministic.
 *
 * Images come as a batch of `batch` equal-shape images stored one after
 * another (image b starts at ptr + b * height * pitch elements). `pitch` is
 * shared by marker, mask, out, grad_out, grad_marker and grad_mask.
 *
 * geo_chain_backward_workspace_size: bytes of device workspace the pair
 *   below needs (checkpoints every ckpt_interval steps, 1 <= ckpt_interval
 *   <= 512; the recomputed states of one segment at every 8th step; the
 *   routing codes of one segment, a 32-bit word per pixel and 8 steps; two
 *   gradient buffers); 0 for invalid arguments.
 * geo_chain_fwd_ckpt: out = the chain of `steps` steps (as geo_dilate_chain /
 *   geo_erode_chain), also storing the checkpoints in `workspace` (caller
 *   owned, ws_bytes >= the size above, else GEO_ERR_WORKSPACE). out must not
 *   alias marker.
 * geo_chain_backward: given the same arguments and the workspace written by
 *   geo_chain_fwd_ckpt (not modified in between), writes grad_marker =
 *   dL/dmarker and grad_mask = dL/dmask for upstream gradient grad_out =
 *   dL/dout. It reuses the workspace's scratch parts but leaves the
 *   checkpoints intact, so a second backward call with the same workspace
 *   is valid. grad buffers must not overlap each other or the inputs.
 */
GEO_API size_t geo_chain_backward_workspace_size(geo_dtype dtype, int64_t height, int64_t width, int64_t steps,
                                         int ckpt_interval, int batch);
GEO_API int geo_chain_fwd_ckpt(geo_dtype dtype, int op, const void *marker, const void *mask, void *out,
                       int64_t height, int64_t width, int64_t pitch, int conn, int64_t steps,
                       int ckpt_interval, int batch, void *workspace, size_t ws_bytes, void *stream);
GEO_API int geo_chain_backward(geo_dtype dtype, int op, const void *mask, const void *grad_out,
                       void *grad_marker, void *grad_mask, int64_t height, int64_t width,
                       int64_t pitch, int conn, int64_t steps, int ckpt_interval, int batch,
                       void *workspace, void *stream);

/*
 * geo_dilate_chain without any memory allocation. The paper has no
 * counterpart; this exists for callers that cannot allocate GPU memory during
 * a call (a fixed memory budget owned by another allocator, a real-time loop
 * that must not reach the driver's allocator, device memory reserved up
 * front). Same arguments and result as geo_dilate_chain; its scratch image is
 * a static device array of 16 MiB that every GPU loading the library holds
 * until the process exits.
 *   - Images whose scratch, round_up(width * element_size, 16) * height bytes,
 *     exceeds 16 MiB are rejected with GEO_ERR_WORKSPACE (4096 x 4096 uint8,
 *     2048 x 2048 float32 and 1448 x 1448 float64 fit).
 *   - All calls share the one array: calls that overlap on the GPU race and
 *     corrupt each other's output; the caller must order them.
 *   - The first call on a device sets up that device (looks up the array's
 *     device address and plans the tiles); make it before any stream capture.
 *   - Every wait of the kernel on another block is bounded. One that expires
 *     leaves out incomplete and records GEO_ERR_TIMEOUT in a status word
 *     inside the static array. The word stays set across later calls until
 *     geo_device_status reads and clears it (that call allocates nothing on
 *     a device where only this entry point has run).
 *   - GEO_ERR_ARG also when the chain needs more than INT_MAX passes.
 */
GEO_API int geo_dilate_chain_noalloc(geo_dtype dtype, const void *marker, const void *mask, void *out,
                             int64_t height, int64_t width, int64_t pitch, int conn,
                             int64_t steps, void *stream);

/*
 * Measurement helper (not part of the method): the rate of the min/max the
 * steps are built from, for the ALU rooflines of the benchmark. form 0:
 * max.u16x2 and form 1: max.f16x2 (the uint8 step, two pixels a lane);
 * form 2: three-input max.f32 (the float32 step's 3-extremes); form 3: a 2:1
 * mix of max.u16x2 with an exact max of u16 lanes computed by two f16
 * instructions on the FMA pipe (each maximum counted once). One block of 1024
 * threads per SM runs 16 independent chains of the instruction per thread;
 * lane_ops_per_clock receives the lane operations retired per SM clock
 * (averaged over the SMs, each SM timed by its own clock counter) and
 * clock_mhz the SM clock over the same span. Synchronous: returns after the
 * probe on `stream` has finished. GEO_ERR_ARG for another form or a NULL
 * output, GEO_ERR_CUDA if a launch, the small allocation or the copy fails.
 */
GEO_API int geo_probe_minmax_rate(int form, double *lane_ops_per_clock, double *clock_mhz, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GEOMORPH_H */
