/*
 * sepconv5.h -- C ABI of libsepconv5, a GB300 (sm_103a) library for the
 * convolution of planar multi-plane images by a separable width-5 kernel
 * (arXiv 1711.09791, "2D Image Convolution using Three Parallel Programming
 * Models on the Xeon Phi").
 *
 * The operation (Eq. 1 of Sec. 1, with the separable matrix K[i][j] = k[i]k[j]):
 *
 *     B[p][y][x] = sum_{a=0..4} sum_{b=0..4} A[p][y+a-2][x+b-2] * k[a] * k[b]
 *
 * evaluated for every plane p and every interior pixel (y, x) with
 * 2 <= y < H-2 and 2 <= x < W-2.  The paper ignores the image edges and starts
 * the convolution at pixel (2,2) (Sec. 5, first paragraph); tap t of k acts at
 * offset t-2 on both axes, with k[0] on the left/top neighbour (Eq. 2 and
 * Listing 1).  It is a correlation: the kernel is not flipped.  Any 5 finite
 * taps are accepted (they need not be symmetric or sum to 1).
 *
 * Two algorithms compute it (Sec. 5.1):
 *   SC5_ALGO_FUSED     single pass: one kernel reads each input pixel from HBM
 *                      once and writes each output pixel once; the horizontal
 *                      pass result stays on chip (the "single-pass without
 *                      copy-back" of Sec. 7, computed as the separable 5+5 form).
 *   SC5_ALGO_TWO_PASS  the horizontal 1D pass writes an FP32 intermediate T to
 *                      HBM, then the vertical 1D pass reads it (Sec. 5.1,
 *                      Listing 1; the horizontal pass covers all H rows so
 *                      that every output row is defined).
 * Both accumulate in FP32 with the taps applied in the order t = 0..4 and give
 * bitwise identical results.
 *
 * Conventions for every call:
 *   - Status codes only; nothing throws across this boundary.  On failure,
 *     sepconv5_last_error() returns a message for the calling thread.
 *   - "dev" pointers are CUDA device pointers of the current device, "host"
 *     pointers are CPU memory.  The caller owns every buffer it passes; a plan
 *     or batch owns only the workspace it allocates itself.
 *   - Image layout is planar: element (p, y, x) of an image with row pitch
 *     `pitch` (in elements) and H rows sits at offset (p*H + y)*pitch + x.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Runs are asynchronous on that stream.
 *   - Sizes: planes >= 1, H >= 5, W >= 5.  For the TMA loads the input base
 *     address must be 16-byte aligned and in_pitch * element size a multiple
 *     of 16 bytes; otherwise SC5_EINVAL.
 *   - Thread safety: distinct plans/batches/servers may be used from
 *     different threads; one plan must not be used by two threads at once.
 */
#ifndef SEPCONV5_H
#define SEPCONV5_H

#include <stddef.h>
#include <stdint.h>

/* Exported symbols keep default visibility when the library is built with
 * -fvisibility=hidden. */
#if defined(__GNUC__)
#define SC5_API __attribute__((visibility("default")))
#else
#define SC5_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SC5_OK = 0,
    SC5_EINVAL = 1,     /* bad argument: sizes, alignment, null pointer, dtype/algo not built */
    SC5_ENOMEM = 2,     /* device or host allocation failed */
    SC5_ECUDA = 3,      /* a CUDA runtime/driver call failed */
    SC5_EAGAIN = 4,     /* serve_submit: queue full (back-pressure); serve_poll: not done yet */
    SC5_ETIMEDOUT = 5,  /* serve_poll: timeout expired before completion */
    SC5_ENOTFOUND = 6,  /* unknown ticket / no tuning entry */
    SC5_EDEVICE = 7     /* a kernel reported a device-side error (a bounded wait ran out) */
} sc5_status;

/* Storage formats.  A stored code c represents the real value value(c)/scale;
 * the scale is a per-image float (1 for F32/BF16/F16 unless the caller says
 * otherwise; for FP8 E4M3 typically 448/max|A|).  Arithmetic is always FP32. */
typedef enum {
    SC5_F32 = 0,        /* IEEE binary32 */
    SC5_BF16 = 1,       /* bfloat16 */
    SC5_F16 = 2,        /* IEEE binary16 */
    SC5_FP8E4M3 = 3     /* OCP FP8 E4M3 (no infinities, max 448); stores saturate */
} sc5_dtype;

typedef enum {
    SC5_BORDER_VALID = 0, /* out is [planes][H-4][out_pitch]; input pixel (2,2) -> out (0,0) */
    SC5_BORDER_KEEP = 1   /* out is [planes][H][out_pitch]; interior as above, the 2-pixel
                             frame is the input converted to the output format (the image
                             Listing 1 leaves behind, computed out of place) */
} sc5_border;

typedef enum {
    SC5_ALGO_FUSED = 0,     /* single pass, separable arithmetic (10 FMA per output) */
    SC5_ALGO_TWO_PASS = 1,  /* horizontal pass to an FP32 intermediate in HBM, then vertical pass */
    SC5_ALGO_DIRECT = 2,    /* single pass, direct form: 25 products per output with the 5x5
                               matrix K (Eq. 1 / Eq. 3); sepconv5_run uses K = k k^T rounded to
                               FP32, sepconv5_run_K takes any K */
    SC5_ALGO_REDUCE = 3     /* one pyramid REDUCE step: the fused result kept at every second row
                               and column.  The paper names convolution and scaling as the two
                               costly steps of its stereo pipeline (Sec. 1) without defining the
                               scaling; this is the blur-then-subsample reading.  Plane p of the
                               output is Ho x Wo with Ho = ceil((H-4)/2), Wo = ceil((W-4)/2),
                               rows out_pitch >= Wo apart, planes Ho*out_pitch apart; output
                               (y, x) is the VALID output (2y, 2x), centred on input (2y+2, 2x+2),
                               bit for bit the SC5_ALGO_FUSED value there.  Planar, width 5,
                               SC5_BORDER_VALID, stacked planes (plane strides 0); every storage
                               pair.  Such a plan runs through sepconv5_run only. */
} sc5_algo;

/* Image layouts.  SC5_LAYOUT_HWC: pixel-interleaved 3-plane images (RGB),
 * value (p, y, x) at y*pitch + 3*x + p for input and output alike (the VALID
 * output row holds 3*(W-4) values); pitches count values.  Built for planes
 * = 3, SC5_ALGO_FUSED, width 5, SC5_BORDER_VALID and every storage pair;
 * in_pitch * element size must be a multiple of 16 bytes. */
typedef enum {
    SC5_LAYOUT_PLANAR = 0,
    SC5_LAYOUT_HWC = 1
} sc5_layout;

/* Plan descriptor.  Pitches and plane strides are in elements of the
 * respective dtype.
 * taps: the kernel width n.  The paper uses 5 (Sec. 4); 3, 7 and 9 are built
 * for SC5_ALGO_FUSED (single image, VALID or KEEP) and then every "5" in this
 * header reads n: k holds n values, tap t acts at offset t-(n-1)/2, the
 * VALID output is (H-n+1) x (W-n+1), the KEEP frame is (n-1)/2 pixels wide,
 * and H, W >= n.  Batches, serving, the two-pass and direct forms, the
 * offload and in-place calls are built for width 5.
 * tile_h/tile_w/stages: 0 = take the autotuned (or built-in default) choice;
 * otherwise one of the compiled fused-kernel shapes (sepconv5_fused_configs).
 * Plane strides: 0 = planes stacked ([planes][H][pitch]: H*in_pitch for the
 * input, Hout*out_pitch for the output).  Any other value places plane p at
 * p*stride; the planes may then be stacked (stride >= H*pitch) or
 * row-interleaved (stride >= W and pitch >= planes*stride), e.g. the 3R x C
 * agglomeration of Sec. 6 where one row holds the rows of all 3 planes side
 * by side: in_pitch = 3*W', in_plane_stride = W'.  The input plane stride
 * times the element size must be a multiple of 16 bytes.  Non-default
 * strides are supported by sepconv5_run, sepconv5_run_K and the two-pass
 * entry points; batches, the offload call and the in-place call take
 * stacked planes. */
typedef struct {
    int32_t planes, H, W;
    int64_t in_pitch, out_pitch;
    int32_t in_dtype, out_dtype;   /* sc5_dtype */
    int32_t border;                /* sc5_border */
    int32_t algo;                  /* sc5_algo */
    int32_t tile_h, tile_w, stages;
    int32_t ctas_per_sm;           /* persistent CTAs per SM, capped at what fits; 0 =
                                      the planner's choice: the tuning table's entry,
                                      else the shape's measured default, else as many
                                      as fit (HWC: as many as fit).  -1: as 0, except
                                      that sepconv5_batch_create times every feasible
                                      count on the batch itself and keeps the fastest
                                      (those launches write the batch's outputs).  -2:
                                      as -1, and every compiled tile shape of the dtype
                                      pair is timed on the batch too (about 0.1 s for
                                      256 images of up to 4096 x 4096) */
    int64_t in_plane_stride, out_plane_stride;
    int32_t taps;                  /* kernel width: 0 or 5 (the paper's), or 3, 7, 9 */
    int32_t layout;                /* sc5_layout */
} sc5_plan_desc;

typedef struct sc5_plan_s *sc5_plan;

/* One image of a batch or one serving request.
 *   in, out: dev pointers for sepconv5_run_batch / sepconv5_batch_create;
 *            host pointers for serve_submit.
 *   H, W, pitches: as in sc5_plan_desc; planes and dtypes come from the plan
 *   (batch) or the server configuration (serve).
 *   k: the 5 taps; in_scale/out_scale: as for sepconv5_run. */
typedef struct {
    const void *in;
    void *out;
    int32_t H, W;
    int64_t in_pitch, out_pitch;
    float k[5];
    float in_scale, out_scale;
} sc5_image;

/* ---------------------------------------------------------------- plans */

/* Validate a descriptor and build a plan for one image shape.  Owns the
 * workspace: the FP32 intermediate T of the two-pass form
 * (planes*H*round_up(W-4,4)*4 bytes, allocated here) and a device status word.
 * Returns SC5_EINVAL for bad sizes/pitches/dtypes, SC5_ENOMEM if the
 * workspace cannot be allocated.  Calls cudaMalloc on the current device. */
SC5_API sc5_status sepconv5_plan(const sc5_plan_desc *desc, sc5_plan *out);
SC5_API sc5_status sepconv5_plan_destroy(sc5_plan plan);
/* The launch configuration a plan chose (from the descriptor, the tuning
 * table or the defaults): fused tile rows and columns, pipeline stages, and
 * CTAs per SM (0 where the kernel takes as many as fit, e.g. HWC plans).
 * Any output pointer may be NULL.  Two-pass plans report the fused shape
 * they would use. */
SC5_API sc5_status sepconv5_plan_info(sc5_plan plan, int32_t *tile_h, int32_t *tile_w, int32_t *stages,
                                      int32_t *ctas_per_sm);

/* Run the plan on one image: in (dev, in_dtype, [planes][H][in_pitch]),
 * out (dev, out_dtype, layout per border), k (host, the plan's taps values --
 * 5 unless the plan says otherwise -- copied by value).  in_scale and
 * out_scale must be finite and > 0; the result code is round(B * out_scale)
 * with B computed from value(in)/in_scale.  `in` and
 * `out` must not overlap.  Asynchronous on `stream`. */
SC5_API sc5_status sepconv5_run(sc5_plan plan, const void *in, void *out, const float k[5],
                        float in_scale, float out_scale, void *stream);

/* Direct single-pass form with a general (not necessarily separable) 5x5
 * matrix: B[p][y][x] = sum_i sum_j A[p][y+i-2][x+j-2] * K[i*5+j] (Eq. 1, the
 * "general algorithm" of Sec. 5.1), summed in FP32 in the row-major order of
 * Eq. 3.  K: host array of 25 finite floats, row-major, copied by value.  The
 * plan must have algo SC5_ALGO_DIRECT; other arguments as for sepconv5_run. */
SC5_API sc5_status sepconv5_run_K(sc5_plan plan, const void *in, void *out, const float K[25],
                                  float in_scale, float out_scale, void *stream);

/* In-place form: `img` (dev, [planes][H][in_pitch], the plan's in_dtype) is
 * replaced by its convolution -- the interior pixels (2 <= y < H-2,
 * 2 <= x < W-2) get the result, the 2-pixel frame keeps its values -- which is
 * the image Listing 1 leaves in A.  The plan must have in_dtype == out_dtype,
 * border SC5_BORDER_KEEP and out_pitch == in_pitch.  A stored code means
 * value(c)/scale before and after.  By algo:
 *   SC5_ALGO_TWO_PASS  Listing 1's structure: horizontal pass img -> T (the
 *                      plan's FP32 intermediate), vertical pass T -> img;
 *   SC5_ALGO_FUSED / SC5_ALGO_DIRECT  the single pass "with copy-back" of
 *                      Sec. 5.2: convolve into a scratch image owned by the
 *                      plan (allocated on the first call), then copy it back.
 * Both move every pixel through HBM twice (the "two assignment operations"
 * of Sec. 7).  Asynchronous on `stream`. */
SC5_API sc5_status sepconv5_run_inplace(sc5_plan plan, void *img, const float k[5], float scale, void *stream);

/* Offload form (the co-processor model of Sec. 7: copy the image to the
 * device, convolve, copy the result back): host_in and host_out are HOST
 * pointers laid out as for sepconv5_run (pinned memory gives full copy
 * bandwidth; pageable memory works but the copies are staged by the driver).
 * The image is cut into bands of rows; the copy of band b+1 to the device,
 * the kernel of band b and the copy of band b-1 back overlap on three
 * streams.  Device staging buffers (input and output image) are allocated by
 * the plan on first use and kept until it is destroyed.  Returns when the
 * result is in host_out; only the output values of each row are written (the
 * row padding of host_out is left as it was).  `stream` carries the kernels. */
SC5_API sc5_status sepconv5_run_host(sc5_plan plan, const void *host_in, void *host_out, const float k[5],
                                     float in_scale, float out_scale, void *stream);

/* Two-pass form, one pass at a time (for checking each pass on its own).
 * hpass writes T (dev, FP32, [planes][H][t_pitch]; t_pitch >= W-4 and a
 * multiple of 4; T 16-byte aligned): column x of row y is the horizontal
 * pass sum_t k[t] * value(in[y][x+t]) centred on input column x+2, for all H
 * rows, on the stored values (not divided by in_scale).  vpass reads such a
 * T and writes `out` exactly as sepconv5_run would. */
SC5_API sc5_status sepconv5_hpass(sc5_plan plan, const void *in, float *T, int64_t t_pitch,
                          const float k[5], void *stream);
SC5_API sc5_status sepconv5_vpass(sc5_plan plan, const float *T, int64_t t_pitch, void *out,
                          const float k[5], float in_scale, float out_scale, void *stream);

/* Two-pass form that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory, such
 * as code running under a framework whose caching allocator owns the GPU's
 * memory, latency-bound loops that cannot absorb the device-wide
 * synchronisation a cudaFree may cause, or plug-ins whose host forbids
 * allocation calls.  It computes exactly what a SC5_ALGO_TWO_PASS plan with
 * SC5_BORDER_VALID computes (same kernels, same bits), but its FP32
 * intermediate lives in a fixed array inside the library instead of a
 * plan's workspace:
 *   - every GPU that loads the library holds that array
 *     (SC5_NOALLOC_MAX_T_FLOATS floats = 16 MiB) until the process exits;
 *   - planes * H * round_up(W-4, 4) must not exceed SC5_NOALLOC_MAX_T_FLOATS
 *     (e.g. 3 planes of 1152 x 1152), else SC5_EINVAL with a message; H <= 65535;
 *   - the first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress, with that device current) and caches it for
 *     the life of the process; make that first call before any stream
 *     capture.  A device reset (cudaDeviceReset) invalidates the cached
 *     address: a process that resets the device must not call this entry
 *     point afterwards;
 *   - it calls no cudaMalloc, cudaFree or other allocating routine;
 *   - all calls share the one array and it keeps the last call's contents;
 *     nothing in it has to start at zero (each call writes every element it
 *     reads), but calls that overlap on the GPU (e.g. on two streams at once)
 *     race on it and must be serialised by the caller.
 * Arguments: in / out are dev pointers laid out as for sepconv5_run with
 * SC5_BORDER_VALID (input 16-byte aligned, in_pitch * element size a
 * multiple of 16); dtype pair, k and scales as for sepconv5_plan /
 * sepconv5_run.  Asynchronous on `stream`. */
#define SC5_NOALLOC_MAX_T_FLOATS 4194304
SC5_API sc5_status sepconv5_two_pass_noalloc(const void *in, void *out, int32_t planes, int32_t H, int32_t W,
                                             int64_t in_pitch, int64_t out_pitch, int32_t in_dtype,
                                             int32_t out_dtype, const float k[5], float in_scale,
                                             float out_scale, void *stream);

/* Synchronise `stream`, then read and clear the device status word shared by
 * every kernel of this library on the current device: 0 if no kernel
 * reported an error since the last call, else SC5_EDEVICE with *code set to
 * the kernel's error code (1 = an mbarrier wait for a TMA load ran out of
 * time). */
SC5_API sc5_status sepconv5_device_status(void *stream, int32_t *code);

/* ---------------------------------------------------------------- pyramids */

/* A multi-scale pyramid: `levels` chained REDUCE steps (SC5_ALGO_REDUCE) of a
 * planar image.  Level 0 is the input ([planes][H][in_pitch], in_dtype);
 * level l >= 1 is the REDUCE step of level l-1, stored in out_dtype (the
 * input's format or SC5_F32) with the library's pitch (rows rounded up to
 * 16 bytes).  The first step converts in_dtype to out_dtype with the given
 * scales; later steps keep out_dtype and its scale.  Every level that is
 * reduced must be at least 5 x 5. */
typedef struct {
    int32_t planes, H, W;
    int64_t in_pitch;          /* elements; in_pitch * element size a multiple of 16 */
    int32_t in_dtype, out_dtype;
    int32_t levels;            /* REDUCE steps, >= 1 */
} sc5_pyramid_desc;

typedef struct sc5_pyramid_s *sc5_pyramid;

/* Validate and build one REDUCE plan per step (no device allocation). */
SC5_API sc5_status sepconv5_pyramid_create(const sc5_pyramid_desc *desc, sc5_pyramid *out);
/* Size of level `level` (0 = the input, 1..levels = the steps' results):
 * rows, columns and row pitch in elements of its format.  A caller allocates
 * level l >= 1 as planes * H * pitch elements. */
SC5_API sc5_status sepconv5_pyramid_level(sc5_pyramid pyr, int32_t level, int32_t *H, int32_t *W,
                                          int64_t *pitch);
/* Run the steps in order on `stream`: in (dev, level 0), levels (host array of
 * `levels` dev pointers, levels[l-1] receives level l, 16-byte aligned), k
 * (host, 5 taps, used at every step).  Asynchronous. */
SC5_API sc5_status sepconv5_pyramid_run(sc5_pyramid pyr, const void *in, void *const *levels, const float k[5],
                                        float in_scale, float out_scale, void *stream);
/* Record sepconv5_pyramid_run for these buffers, taps and scales into a
 * CUDA graph kept by the pyramid (replacing any earlier one), so that the
 * small levels cost no per-launch host work: sepconv5_pyramid_replay then
 * runs it on `stream`.  The buffers must stay valid and keep their addresses
 * while the graph is used.  Nothing runs at capture time. */
SC5_API sc5_status sepconv5_pyramid_capture(sc5_pyramid pyr, const void *in, void *const *levels, const float k[5],
                                            float in_scale, float out_scale);
SC5_API sc5_status sepconv5_pyramid_replay(sc5_pyramid pyr, void *stream);
SC5_API sc5_status sepconv5_pyramid_destroy(sc5_pyramid pyr);

/* ---------------------------------------------------------------- batches */

/* Run many images of different sizes and kernels in one persistent launch
 * driven by a tile work-list.  The plan supplies planes, dtypes, border and
 * algo (must be SC5_ALGO_FUSED); its H/W are ignored.  imgs is a host array of
 * n images whose in/out are dev pointers.  Builds the work-list and the
 * per-image TMA descriptors on the host, uploads them to workspace owned by
 * the plan (grown as needed, stream-ordered) and launches.  The tile shape is
 * taken from the plan's override or from the autotuner for the batch's
 * dominant size class. */
SC5_API sc5_status sepconv5_run_batch(sc5_plan plan, int32_t n, const sc5_image *imgs, void *stream);

/* A prepared batch: work-list and descriptors uploaded once, the launch
 * captured in a CUDA graph.  sepconv5_batch_launch replays it on `stream`
 * (the images' buffers must stay valid and keep their addresses). */
typedef struct sc5_batch_s *sc5_batch;
SC5_API sc5_status sepconv5_batch_create(sc5_plan plan, int32_t n, const sc5_image *imgs,
                                 sc5_batch *out);
SC5_API sc5_status sepconv5_batch_launch(sc5_batch batch, void *stream);
/* Number of tiles and of CTAs of the prepared launch (for reporting). */
SC5_API sc5_status sepconv5_batch_info(sc5_batch batch, int64_t *tiles, int32_t *ctas,
                               int32_t *tile_h, int32_t *tile_w);
SC5_API sc5_status sepconv5_batch_destroy(sc5_batch batch);

/* ---------------------------------------------------------------- tuning */

/* Compiled fused-kernel shapes for an (in, out) dtype pair: writes up to
 * `cap` triples (tile_h, tile_w, stages) into cfg and their count to *n. */
SC5_API sc5_status sepconv5_fused_configs(int32_t in_dtype, int32_t out_dtype, int32_t *cfg,
                                  int32_t cap, int32_t *n);

/* Autotuner (the counterpart of the paper's thread/task-count tuning, Sec. 4
 * and Sec. 7): for every size class (log2 of the plane area, 7 classes from
 * below 2^14 to 2^24 pixels and above), dtype pair in `dtypes` (pairs in, out)
 * and kernel kind (the single-image kernel of plans; the work-list kernel of
 * batches and merged serving launches), time every compiled shape and CTA
 * count on synthetic images on the current device and keep the fastest.
 * mode: 0 = off (clears the table: built-in defaults), 1 = quick (3
 * repetitions per configuration), 2 = full (10 repetitions).  The table is kept in the process and, if path is
 * not NULL, written there as JSON keyed by GPU name.  Allocates device memory
 * for its test images. */
SC5_API sc5_status sepconv5_autotune(int32_t mode, const int32_t *dtypes, int32_t n_pairs,
                             const char *path);
/* The same from the environment, without code changes, once per dtype pair on
 * the pair's first plan, batch or server in the process:
 *   SEPCONV5_TUNE_FILE=path   load a table written by sepconv5_autotune, and
 *                             write the table back there after tuning;
 *   SEPCONV5_TUNE=quick|full  tune the pair (modes 1 and 2 above) unless the
 *                             table already holds all of its entries; that
 *                             call then takes a few seconds;
 *   SEPCONV5_TUNE=off or unset: built-in defaults unless a table is loaded.
 * Failures leave the defaults in place. */
/* Load a table written by sepconv5_autotune (entries for other GPUs are ignored). */
SC5_API sc5_status sepconv5_tune_load(const char *path);
/* The shape a plan would pick for a plane of H x W with these dtypes:
 * SC5_OK with the tuned entry, or SC5_ENOTFOUND with the default shape and
 * ctas_per_sm = 0 when the table has none. */
SC5_API sc5_status sepconv5_tune_lookup(int32_t in_dtype, int32_t out_dtype, int32_t H, int32_t W,
                                int32_t *tile_h, int32_t *tile_w, int32_t *stages,
                                int32_t *ctas_per_sm);
/* The same for a batch (or merged serving launch) whose dominant size class
 * is that of an H x W plane. */
SC5_API sc5_status sepconv5_tune_lookup_batch(int32_t in_dtype, int32_t out_dtype, int32_t H, int32_t W,
                                      int32_t *tile_h, int32_t *tile_w, int32_t *stages,
                                      int32_t *ctas_per_sm);

/* ---------------------------------------------------------------- serving */

typedef struct sc5_server_s *sc5_server;

typedef struct {
    size_t hbm_budget_bytes;  /* device bytes for resident request buffers */
    int32_t max_inflight;     /* requests admitted and not yet completed */
    int32_t dtype;            /* storage format of inputs and outputs */
    int32_t planes;           /* planes per image */
    int32_t n_streams;        /* compute streams used round robin (>= 1) */
    int32_t max_merge;        /* most requests merged into one launch (0 = no limit) */
    int32_t merge;            /* 1 = continuous batching, 0 = one launch per request */
    int32_t batch_window_us;  /* hold admitted requests up to this long (or until max_merge
                                 are waiting) before launching them together; 0 = launch
                                 whatever one pass of the scheduler admitted at once */
} sc5_serve_cfg;

typedef struct {
    uint64_t submitted, completed, launches, rejected;
    uint64_t merged_max;         /* largest number of requests in one launch */
    size_t resident_peak_bytes;  /* high-water mark of admitted buffers */
    /* Where completed requests spent their time (microseconds, host clock,
     * median and 99th percentile over the last 2^20 completions; 0 before the
     * first):  queue = submitted until admitted (waiting for arena space or an
     * in-flight slot);  stage = admitted until its launch is enqueued (the
     * input copy is enqueued at admission; a batching window adds its wait);
     * run = launch enqueued until the completion thread sees the request's
     * output copy done (input copy still in flight, kernel, output copy). */
    double queue_us_p50, queue_us_p99, stage_us_p50, stage_us_p99, run_us_p50, run_us_p99;
} sc5_serve_stats;

/* Start a server on the current device: allocates its resident arena
 * (hbm_budget_bytes), warms it up (the arena is written once, every compiled
 * batch-kernel shape of the dtype is loaded, events are created up front, so
 * that the first requests run as fast as later ones; this takes a few
 * milliseconds and waits for the arena writes) and starts its scheduler and
 * completion threads.
 * Host-side fault injection for tests, read from the environment here:
 * SC5_SERVE_FAULT=arena_alloc makes the arena allocation fail (SC5_ENOMEM);
 * SC5_SERVE_FAULT=sched_delay_ms=N makes the scheduler sleep N ms before
 * each admission round.  Neither touches the GPU. */
SC5_API sc5_status serve_create(const sc5_serve_cfg *cfg, sc5_server *out);

/* Queue one request.  req->in and req->out are HOST pointers to
 * [planes][H][pitch] images of the server's dtype, in page-locked memory
 * (cudaMallocHost, cudaHostAlloc or cudaHostRegister); the server reads `in`
 * and writes the W-4 output values of each row of `out` (its row padding is
 * left as it was) asynchronously, so both must stay valid until serve_poll
 * returns SC5_OK for the ticket.  The output buffer is named here rather
 * than at serve_poll: its copy is issued behind the kernel as soon as the
 * request is launched, and lands while the caller is not yet polling.
 * A request that fits the budget but not the arena's free space waits in the
 * queue until earlier requests retire.  Returns SC5_EAGAIN when 65536
 * requests are already queued (back-pressure: retry later), SC5_EINVAL for a
 * bad shape, non-finite taps, a scale that is not finite and > 0, a host
 * buffer that is not page-locked, or a request that needs more than the
 * whole budget. */
SC5_API sc5_status serve_submit(sc5_server srv, const sc5_image *req, uint64_t *ticket);

/* Wait up to timeout_us (0 = just test, <0 = forever) for a ticket.  SC5_OK:
 * the output is in req->out and *latency_us (if not NULL) holds the time from
 * submit to completion of the device-to-host copy; the ticket is retired.
 * SC5_EAGAIN (timeout_us == 0) or SC5_ETIMEDOUT: not done yet. */
SC5_API sc5_status serve_poll(sc5_server srv, uint64_t ticket, int32_t timeout_us, double *latency_us);

SC5_API sc5_status serve_get_stats(sc5_server srv, sc5_serve_stats *stats);

/* Drain every queued and in-flight request, stop the threads, free the arena. */
SC5_API sc5_status serve_destroy(sc5_server srv);

/* ---------------------------------------------------------------- misc */

/* Message for the last failing call on this thread ("" if none). */
SC5_API const char *sepconv5_last_error(void);

/* Launch an empty kernel `n` times on `stream` (the launch-overhead probe, the
 * counterpart of the paper's empty-kernel measurement in Sec. 6). */
SC5_API sc5_status sepconv5_empty_launches(int32_t n, void *stream);

/* Failure-path self-test: launch one warp that waits, with the same bounded
 * mbarrier wait the fused kernels use, on a barrier that nothing completes.
 * After limit_us (1..100000) of GPU time it writes error code 1 into the
 * device status word and exits normally -- no trap, no fault; the context
 * stays usable.  A following sepconv5_device_status then reports SC5_EDEVICE
 * with code 1 (and clears it). */
SC5_API sc5_status sepconv5_selftest_wait_timeout(int32_t limit_us, void *stream);

/* Number of kernels this library launched in this process (all entry points). */
SC5_API int64_t sepconv5_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SEPCONV5_H */
