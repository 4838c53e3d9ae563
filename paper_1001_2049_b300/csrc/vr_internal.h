// vr_internal.h -- declarations shared by the host API and the CUDA kernels
// of libvr.  Not part of the public ABI (include/vr.h is).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "vr.h"

namespace vr {

constexpr int kBrick = VR_BRICK;                  // 32
constexpr int kBrickShift = 5;
constexpr int64_t kBrickVoxels = 32 * 32 * 32;    // 32768
constexpr int kMaxViewsPerLaunch = 64;            // cameras travel as kernel parameters
constexpr int kMaxLayers = 2048;                  // layers of a layered texture
// Texel formats of texture storage, also the storage codes the texture
// kernels are specialised on: the plain storage types (VR_F32, VR_F16, VR_I8:
// one voxel per texel) and the pair formats, where a texel packs a voxel with
// its neighbour in the next frequency plane (two binary16 in 32 bits, or two
// int8 codes, each plus 128, in 16 bits), so one gather returns all eight
// corners of a cell.
constexpr int kF16Pair = 3;
constexpr int kI8Pair = 4;
// Empty-space masks: per macrocell of 4 x 4 x 4 cells, a 64-bit mask of the
// cells that a clip level leaves visible (bit (x & 3) | (y & 3) << 2 |
// (z & 3) << 4).  Cells are indexed by their gather coordinates: on every
// axis cells -1 .. n - 1 stored at cell + 1 (the outermost ones hold
// positions a rounding error outside the box, which read the edge voxels).
constexpr int kMacroShift = 2;
constexpr int kMacro = 1 << kMacroShift;

// MIP bounds: every voxel v is stored as an 8-bit code c with L + c delta >=
// v (exact arithmetic), two planes per 16-bit texel (cell slices, as the pair
// formats), one code scale for the whole cube.  The march tests a sample by
// the trilinear value of its cell's codes, each read as the float
// 1 + c 2^-15, against a limit derived from the ray's running maximum
// (vr_ray.cuh, bound_limit).  This device record holds the scale and the
// limit's constants; vr_tex.cu derives them from the cube's smallest and
// largest finite voxels (reduced into lo / hi as ordered bit patterns) and
// sets le = +inf, which makes every sample a candidate, when the cube holds
// +inf, its range is not finite, or a later fill meets a voxel the scale
// does not cover.
struct BoundScale {
    float L, delta;         // code c stands for L + c delta, c in [0, 255]
    float le, inv_q;        // bound_limit: (m - le) inv_q + 1 - 2^-19, rounded down
    float vlim;             // largest |voxel| le's rounding term covers
    unsigned lo, hi;        // ordered bit patterns of the smallest / largest finite voxel
    unsigned inf;           // nonzero: a +inf voxel was seen
};

// Geometry of a bricked volume, as the kernels see it.
struct VolumeGeom {
    int nx, ny, nz;         // voxel dims
    int nbx, nby, nbz;      // brick counts per axis
};

// Host-side volume handle.
struct Volume {
    VolumeGeom g;
    int dtype;
    void* bricks;           // caller-owned device buffer (null once dropped)
    size_t bytes;
    bool texture_only;      // bricks dropped: the texture is the only copy
    float* scale;           // VR_I8: per-plane tables inside the buffer
    float* offset;
    // transfer function as set by the user
    float lut_raw[VR_MAX_LUT][4];
    int n_lut;
    float v_lo, v_hi, clip, term_alpha;
    // opacity-corrected table cache (depends on the step)
    float lut_step;
    float lut_corr[VR_MAX_LUT][4];
    bool lut_valid;
    // optional texture storage (library-owned): one layered 2-D texture,
    // one plane (plain formats) or cell plane (pair formats) per 2-D slice,
    // 2^stack_shift slices stacked per layer
    bool has_tex;
    int tex_format;         // VR_F32 / VR_F16 / VR_I8, or kF16Pair / kI8Pair
    cudaArray_t array;      // nz + 2 slices (plain) or nz + 1 (pair), see vr_ray.cuh
    cudaTextureObject_t tex;
    int stack_shift;        // 0: a layer per slice
    int stack_pitch;        // rows per stacked slice (ny + 2) when stacked
    void* dec;              // VR_I8: per-slice decode records (library-owned)
    // optional MIP bounds (VR_F32 with texture storage, library-owned): cell
    // slices as the pair formats (slice s packs planes s - 1 and s), every
    // voxel as an 8-bit upper-bound code (BoundScale), stacked as the texture
    cudaArray_t bound_array;
    cudaTextureObject_t bound_tex;
    BoundScale* bound_scale;    // device record of the code scale
    int cfg[3];             // texture-kernel launch shape per mode (autotuned)
    // optional empty-space masks (caller-owned device buffer)
    unsigned long long* mask;   // valid for clip level mask_clip
    float mask_clip;            // NaN: not built
    int mnx, mny, mnz;          // macrocells per axis
};

// Texture storage as the texture kernels see it.
// int8 texture storage decodes with its planes' scales and offsets, read per
// texture slice from one record: plain int8 slice s -> {scale, offset} of
// plane s - 1 (clamped); pair slice s -> {scale, scale, offset, offset} of
// planes s - 1 and s (clamped); applied to each plane's bilinear value of
// the codes (interp_t).
struct TexParams {
    cudaTextureObject_t tex;
    int stack_shift, stack_pitch;   // see Volume
    const void* dec;        // VR_I8 / kI8Pair: float2 / float4 per slice
    int k_max;
    // MIP bounds (0: none): 8-bit upper-bound codes of the FP32 voxels, two
    // planes per 16-bit texel in cell slices (as the pair formats), with
    // `tex`'s stacking, and their scale (BoundScale); a sample whose bound
    // stays below the limit derived from the ray's running maximum cannot
    // raise it (see march_tex_bound)
    cudaTextureObject_t bound;
    const BoundScale* bound_scale;
};

size_t brick_bytes(const VolumeGeom& g, int dtype);   // voxel part only
size_t table_offset(const VolumeGeom& g, int dtype);  // where VR_I8 tables start

// Kernel parameters of one march launch (passed by value; ~8.6 KB).
struct MarchParams {
    const void* bricks;
    const float* scale;     // VR_I8 only
    const float* offset;
    VolumeGeom g;
    float hix, hiy, hiz;    // n - 1 per axis
    int w, h, n_views;
    float step;
    float clip, term_alpha;
    float v_lo, lut_scale;  // x = (s - v_lo) * lut_scale, lut_scale = (N-1)/(v_hi-v_lo)
    float lut_max;          // N - 1
    int n_lut;
    float* out;             // first view of this launch
    unsigned long long* samples;   // may be null
    const unsigned long long* mask;   // empty-space masks for `clip` (COMPOSITE), or null
    int mnx, mny, mlast;              // macrocells along x, y; last macrocell index
    // rendering one part of a larger cube (vr_render_part): the cells of the
    // part, the part's first plane, which rays (+1 going up, -1 going down)
    int part_lo, part_hi, slice_base, sweep;
    vr_camera cams[kMaxViewsPerLaunch];
    float4 lut[VR_MAX_LUT];
};

// ---- batched persistent launch ----
constexpr int kMaxBatch = VR_BATCH_MAX;        // requests per launch
constexpr int kMaxBatchTex = 8;                // textured volumes per launch
constexpr int kMaxBatchLut = 2;                // distinct corrected tables per launch
// Workspace words of one launch: the work counter and one tile counter per
// request.
constexpr int kBatchWords = 1 + kMaxBatch;

struct BatchTex {
    cudaTextureObject_t tex;
    int stack_shift, stack_pitch;   // see Volume
    int format;            // texel format (see kF16Pair)
    const void* dec;       // as TexParams::dec
};

// One request as the batched kernel sees it (field names shared with
// MarchParams so the per-ray march templates accept either).
struct BatchReq {
    vr_camera cam;
    float* out;
    const void* bricks;
    const float* scale;
    const float* offset;
    unsigned long long* samples;
    unsigned* done;
    const unsigned long long* mask;   // empty-space masks, or null
    int mnx, mny;
    VolumeGeom g;
    float hix, hiy, hiz, step;
    float clip, term_alpha, v_lo, lut_scale, lut_max;
    int w, h, n_lut, k_max, mode, dtype;
    int tex_slot;          // -1: gather from the bricks
    int lut_slot;
    int tiles_x, n_tiles, first_item;
    int row0, row_end;     // the image rows rendered; `out` starts at row0
    unsigned done_value;
};

struct BatchParams {
    int n, total_items;
    BatchReq req[kMaxBatch];
    BatchTex tex[kMaxBatchTex];
    float4 lut[kMaxBatchLut][VR_MAX_LUT];
};

// Launch classes of the batched kernel, each compiled as its own kernel:
// requests on volumes without texture storage, on volumes with plain texel
// formats and with pair texels (which need fewer registers, so that class
// keeps more warps resident).
enum BatchClass { kBatchBricks = 0, kBatchTex = 1, kBatchTexPair = 2, kNumBatchClasses = 3 };
// Tile and ray-packet shapes of the batched kernel (the batch autotuner's
// search space): a tile of tx x ty rays (one block of 256 threads) whose
// warps hold px x py packets of neighbouring rays.
struct BatchShape {
    int tx, ty, px, py;
};
constexpr BatchShape kBatchShapes[] = {
    {16, 16, 8, 4}, {16, 16, 16, 2}, {16, 16, 4, 8}, {32, 8, 8, 4}, {32, 8, 16, 2}, {64, 4, 16, 2},
};
constexpr int kNumBatchShapes = sizeof(kBatchShapes) / sizeof(kBatchShapes[0]);
cudaError_t launch_batch(const BatchParams& b, unsigned* ws, int grid, int cls, int cfg,
                         cudaStream_t s);
int batch_blocks_per_sm(int cls, int cfg);
int batch_with_counters(const vr_request* reqs, int n, unsigned* counters, cudaStream_t s);
int record_error(int code, const char* msg);

// Shape of the shared-memory window of the slab-staged march.
struct SlabConfig {
    int S;          // cells per slab along the principal axis (S + 1 planes staged)
    int margin;     // voxels added around the reduced window on each side
    int eb_max;     // window capacity along the innermost axis (multiple of 4)
    int ec_max;     // window capacity along the third axis
    int ea_pitch;   // plane pitch when x is the principal axis (>= S + 1, odd)
    int k_max;      // bound on samples per ray
    int win_elems;  // elements of one window buffer (two are allocated)
    float min_axis; // slab along y/z when that component of the direction is at least this
    size_t smem_bytes;
};

// Launchers (return a cudaError_t from the launch).
cudaError_t launch_march(const MarchParams& p, int dtype, int mode, cudaStream_t s);
cudaError_t launch_slab(const MarchParams& p, const SlabConfig& c, int mode, cudaStream_t s);
size_t slab_smem_bytes(const SlabConfig& c);
size_t slab_window_elems(const SlabConfig& c);
// Window shape for the cameras of one launch (false: use the gather kernel).
bool plan_slab(const MarchParams& p, SlabConfig* c);
cudaError_t launch_tex(const MarchParams& p, const TexParams& t, int format, int mode, int cfg,
                       cudaStream_t s);
// Render one part of a larger cube, continuing the images in p.out.
// Scene integration of sub-cubes' partial images (vr_integrate.cu).
struct IntegrateParams {
    const float* partials;   // the views' first pixel in sub-cube 0's partial images
    float* out;
    size_t part_stride;      // pixels from one sub-cube's partial images to the next's
    int n_parts, n_views, w, h;
    vr_camera cams[kMaxViewsPerLaunch];
};
cudaError_t launch_integrate(const IntegrateParams& p, int mode, cudaStream_t s);
// Object-order MIP (vr_object.cu): one block per sub-cube of 32^3 cells,
// adding each ray's partial maxima to `p.out` (filled with -inf first).
cudaError_t launch_object(const MarchParams& p, int k_max, int dtype, cudaStream_t s);

cudaError_t launch_part(const MarchParams& p, const TexParams& t, int format, int mode,
                        cudaStream_t s);
cudaError_t launch_part_f32(const MarchParams& p, const TexParams& t, int mode, cudaStream_t s);
cudaError_t launch_part_f16(const MarchParams& p, const TexParams& t, int mode, cudaStream_t s);
cudaError_t launch_part_i8(const MarchParams& p, const TexParams& t, int mode, cudaStream_t s);
cudaError_t launch_part_f16pair(const MarchParams& p, const TexParams& t, int mode,
                                cudaStream_t s);
cudaError_t launch_part_i8pair(const MarchParams& p, const TexParams& t, int mode,
                               cudaStream_t s);
// Fill n_pixels images with the empty state of `mode` (0 / -inf / 0).
cudaError_t launch_render_init(float* out, size_t n_pixels, int mode, cudaStream_t s);
// One texel format each (vr_tex_<format>.cu).
cudaError_t launch_tex_f32(const MarchParams& p, const TexParams& t, int mode, int cfg,
                           cudaStream_t s);
cudaError_t launch_tex_f16(const MarchParams& p, const TexParams& t, int mode, int cfg,
                           cudaStream_t s);
cudaError_t launch_tex_i8(const MarchParams& p, const TexParams& t, int mode, int cfg,
                          cudaStream_t s);
cudaError_t launch_tex_f16pair(const MarchParams& p, const TexParams& t, int mode, int cfg,
                               cudaStream_t s);
cudaError_t launch_tex_i8pair(const MarchParams& p, const TexParams& t, int mode, int cfg,
                              cudaStream_t s);
// Empty-space masks of every macrocell for clip level `clip`.
cudaError_t launch_masks(const Volume& v, float clip, cudaStream_t s);
int tex_shape_count();
void tex_shape(int cfg, int* bx, int* by, int* px, int* py, int* minb);
// Per-slice int8 decode records of the volume's texture (see TexParams).
cudaError_t fill_decode_records(const Volume& v, cudaStream_t s);
// Fill texture slices [s0, s1) from the bricks through surface `surf`.
cudaError_t fill_texture(const Volume& v, cudaSurfaceObject_t surf, int s0, int s1,
                         cudaStream_t s);
// The MIP bounds' code scale of the whole cube (VR_F32 bricks): reset
// v.bound_scale, reduce the smallest and largest finite voxel into it and
// derive the scale and the march's constants.
cudaError_t bound_scale(const Volume& v, cudaStream_t s);
// Fill MIP-bound cell slices [s0, s1) (VR_F32 bricks: slice s packs the codes
// of planes s - 1 and s, clamped) through `surf`; a voxel above the scale's
// cap turns skipping off (BoundScale).
cudaError_t fill_bounds(const Volume& v, cudaSurfaceObject_t surf, int s0, int s1,
                        cudaStream_t s);
// The same slices written linearly (x fastest, slice after slice) to `dst`,
// for a copy into an unstacked bound texture.
cudaError_t fill_bounds_linear(const Volume& v, unsigned short* dst, int s0, int s1,
                               cudaStream_t s);
cudaError_t launch_pack(const Volume& v, int64_t z0, int64_t nplanes, const float* src,
                        cudaStream_t s);
// The checked build (VR_DEBUG): the failed-check bits each translation unit
// with checked kernels recorded (read, and cleared when `clear`); 0 in other
// builds.
unsigned debug_flags_tex_f32(bool clear);
unsigned debug_flags_tex_f16(bool clear);
unsigned debug_flags_tex_i8(bool clear);
unsigned debug_flags_tex_f16pair(bool clear);
unsigned debug_flags_tex_i8pair(bool clear);
unsigned debug_flags_batch(bool clear);
unsigned debug_flags_integrate(bool clear);
unsigned debug_flags_object(bool clear);

}  // namespace vr
