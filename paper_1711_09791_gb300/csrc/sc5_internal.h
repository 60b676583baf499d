// sc5_internal.h -- declarations shared by the translation units of
// libsepconv5 (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/sepconv5.h"

namespace sc5 {

constexpr int kTaps = 5;
constexpr int kHalo = 4;          // a width-5 kernel needs 2 extra pixels per side
constexpr int kMaxTaps = 9;       // widest kernel the fused separable path is built for
constexpr int kColsPerThread = 4; // output columns per consumer thread

// Error codes written to the device status word.
constexpr int kDevErrTmaTimeout = 1;

// Per-image description read by the fused kernels.  The tensor map describes
// the input image as a 3-D tensor (x = column, y = row, z = plane).
struct alignas(128) ImgDesc {  // CUtensorMap's own alignment
    CUtensorMap tmap;      // 128 bytes
    void *out;             // first VALID output pixel (plane 0)
    int64_t out_pitch;     // elements
    int64_t out_plane;     // elements between planes
    int32_t Hv, Wv;        // VALID output rows / cols
    int32_t tiles_x, tiles_y;
    float k[kMaxTaps];     // taps (the first `taps` entries are used)
    float oscale;          // out_scale / in_scale
    int32_t vec;           // 1: 4-wide vector stores are aligned
    float K[kTaps * kTaps];  // direct form: the 5x5 matrix, row-major, K[i][j] at offset (i-2, j-2)
    int32_t pad_[8];
};
static_assert(sizeof(ImgDesc) == 384, "ImgDesc: 128-byte tensor map + 216 bytes of parameters, padded to 128");

// One entry of a batch work-list: a (th x tw) output tile of one plane.
struct TileRec {
    int32_t img, plane, ty, tx;
};

// A compiled fused-kernel shape.
struct FusedShape {
    int tile_h, tile_w, rows_per_thread, stages;
};

// Fused kernel launchers (sc5_fused.cu).  Return a cudaError_t.  `direct`
// selects the direct single-pass kernels (25 products per output, K from the
// descriptor); they have their own shape list.
// `taps` (3, 5, 7 or 9) selects the separable kernels of that width (5 for
// the direct kernels).
int fused_num_shapes(int in_dtype, int out_dtype, bool direct = false, int taps = 5);
bool fused_shape(int in_dtype, int out_dtype, int idx, FusedShape *s, bool direct = false, int taps = 5);
int fused_find_shape(int in_dtype, int out_dtype, int tile_h, int tile_w, int stages, bool direct = false,
                     int taps = 5);
// Threads per CTA of a shape.
int fused_threads(const FusedShape &s);
// Max resident CTAs per SM for a shape (occupancy query), or <= 0 on error.
int fused_max_ctas_per_sm(int in_dtype, int out_dtype, int idx, bool direct = false, int taps = 5);
// CTAs per SM a shape runs when no tuning entry or descriptor names one (0: as many as fit).
int fused_default_ctas(int in_dtype, int out_dtype, int idx, bool direct = false, int taps = 5);
// Set the kernel attributes of a shape on the current device (call before
// capturing a launch into a graph).
cudaError_t fused_prepare(int in_dtype, int out_dtype, int idx, bool direct = false, int taps = 5);
cudaError_t launch_fused_single(int in_dtype, int out_dtype, int idx, const ImgDesc &d,
                                int64_t ntiles, int grid, cudaStream_t st, bool direct = false, int taps = 5);
cudaError_t launch_fused_batch(int in_dtype, int out_dtype, int idx, const ImgDesc *descs,
                               const TileRec *tiles, int64_t ntiles, int grid, cudaStream_t st);
cudaError_t read_and_clear_device_status(cudaStream_t st, int32_t *code);
cudaError_t launch_wait_selftest(int limit_us, cudaStream_t st);
int *status_word();  // device address of the status word on the current device

// Pixel-interleaved (HWC, 3 planes) fused kernel (sc5_hwc.cu).
int hwc_box_cols(int in_dtype);              // values per TMA box row
int hwc_tile_h(int in_dtype, int out_dtype); // output rows per tile (0: pair not built)
size_t hwc_desc_size();
void hwc_fill(void *desc, const CUtensorMap &m, void *out, int64_t out_pitch, int Hv, int Wv, int tile_h,
              const float *k, float oscale, bool vec);
// Pyramid REDUCE kernel (sc5_reduce.cu): the compiled shape with tile_h input
// rows per tile and `stages` stages (tile_h 0: the default; stages 0: any),
// false if none; and its launcher.  desc.Hv / desc.Wv hold the output extents
// and desc.tiles_x / desc.tiles_y the grid of TH x 128 input tiles.
bool reduce_shape(int in_dtype, int out_dtype, int tile_h, int stages, FusedShape *sh);
cudaError_t launch_reduce(int in_dtype, int out_dtype, const FusedShape &sh, const ImgDesc &desc, int64_t ntiles,
                          int ctas_per_sm, cudaStream_t st);
// ctas_per_sm <= 0 or above what fits: as many CTAs per SM as fit.
cudaError_t launch_hwc(int in_dtype, int out_dtype, const void *desc, int64_t ntiles, int ctas_per_sm, cudaStream_t st);

// Two-pass kernels and helpers (sc5_twopass.cu).
cudaError_t launch_hpass(int in_dtype, const void *in, int P, int H, int W, int64_t in_pitch,
                         float *T, int64_t t_pitch, const float *k, cudaStream_t st, int64_t in_plane = 0);
cudaError_t launch_vpass(int out_dtype, const float *T, int P, int H, int Wv, int64_t t_pitch,
                         void *out, int64_t out_pitch, int64_t out_plane, const float *k,
                         float oscale, bool vec, cudaStream_t st);
cudaError_t launch_keep_frame(int in_dtype, int out_dtype, const void *in, int P, int H, int W,
                              int64_t in_pitch, void *out, int64_t out_pitch, float ratio,
                              cudaStream_t st, int64_t in_plane = 0, int64_t out_plane = 0, int radius = 2);
cudaError_t launch_empty(int n, cudaStream_t st);
// Copy a VALID image into an interior that starts 2 elements into its rows
// (src rows 16-byte aligned, dst interior 2*element-size aligned).
cudaError_t launch_copy_interior(int dtype, const void *src, int64_t src_pitch, int64_t src_plane, void *dst,
                                 int64_t dst_pitch, int64_t dst_plane, int P, int rows, int cols, cudaStream_t st);

// Library-wide helpers (sc5_api.cu).
void note_launches(int64_t n);
int dtype_bytes(int dtype);
int num_sms();
sc5_status fail(sc5_status st, const char *fmt, ...);
sc5_status fail_cuda(cudaError_t e, const char *what);
void clear_error();
// Fused shape and CTAs/SM for a plane size (override > tuned table > default);
// `batch` selects the tuning entries of the work-list kernel (batches, merged
// serving launches) instead of those of the single-image kernel.
sc5_status choose_shape(int in_dtype, int out_dtype, int H, int W, const sc5_plan_desc *ov, int *idx, int *ctas,
                        bool direct = false, int taps = kTaps, bool batch = false);
// Shape for a set of images: tuned choice for the size class with most pixels.
sc5_status choose_batch_shape(int in_dtype, int out_dtype, int n, const sc5_image *imgs, int *idx, int *ctas);
// Host image of a batch launch: ImgDesc[n] then (256-byte aligned) TileRec[tiles].
sc5_status build_batch(const sc5_plan_desc &pd, int n, const sc5_image *imgs, const FusedShape &sh,
                       std::vector<unsigned char> *blob, int64_t *ntiles, size_t *tiles_off);

}  // namespace sc5
