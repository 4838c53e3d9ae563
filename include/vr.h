/*
 * vr.h -- C ABI of libvr, a ray caster for noisy RA x Dec x frequency
 * spectral cubes on NVIDIA B300 (sm_103a).
 *
 * The operation (paper §3.1, process item 3): every output pixel is mapped
 * to one ray through the cube, and the ray to a colour plus opacity (RGBA)
 * through a pre-selected transfer function, or to a maximum-intensity value.
 * The paper states the problem, not the arithmetic; the arithmetic this
 * library implements is:
 *
 *   camera -> ray   u = px + 1/2 - w/2, v = py + 1/2 - h/2 (pixel centres);
 *                   VR_ORTHO: origin eye + u du + v dv, direction fwd/|fwd|;
 *                   VR_PERSP: origin eye, direction (fwd + u du + v dv)/|..|.
 *   ray / box       box [0, n-1] on each axis (voxel centres at integers);
 *                   slab test, an axis the ray is parallel to passes iff the
 *                   origin lies within [0, n-1] on it.  t_entry = max(0,
 *                   largest near distance), t_exit = smallest far distance.
 *   samples         K = floor((t_exit - t_entry)/step) + 1 when the ray hits;
 *                   sample k sits at t_entry + k*step (from the integer k,
 *                   never an accumulated t), clamped to the box.
 *   trilinear       i0 = min(floor(p), n-2), f = p - i0 per axis; the eight
 *                   corners are interpolated along x, then y, then z.
 *   transfer fn.    (paper abstract: special attention to low signal-to-
 *                   noise data) samples below `clip` are fully transparent;
 *                   others are looked up, with linear interpolation, in an
 *                   RGBA table spanning [v_lo, v_hi] whose opacities are per
 *                   unit voxel length and are corrected to the step as
 *                   alpha' = 1 - (1 - alpha)^step.
 *   VR_COMPOSITE    front to back: C += (1-A) alpha rgb, A += (1-A) alpha; a
 *                   ray stops after the first composited sample with
 *                   A >= term_alpha.  Output premultiplied RGBA, 0 on a miss.
 *   VR_MIP          maximum sample value (raw data units), -inf on a miss.
 *   VR_SUM          sum of sample * step (an additive mode for testing).
 *
 * Arithmetic is single precision with FP32 accumulation whatever the
 * storage type.
 *
 * Memory.  The caller owns the device memory a render reads and writes: the
 * brick buffer of each volume (size from vr_volume_bytes), the empty-space
 * masks, every source, output buffer and batch workspace.  The library owns
 * the small host-side handle and, when asked for them, a volume's texture
 * storage and MIP bounds (vr_volume_attach_texture,
 * vr_volume_attach_mip_bounds: the device allocations it makes, besides a
 * stream-ordered scratch buffer while bounds are filled).  Every call that
 * takes a stream (a cudaStream_t passed as void*, NULL = legacy default
 * stream) is asynchronous on it: argument errors are reported synchronously;
 * a device fault surfaces at the caller's next synchronisation.  The library
 * never synchronises on its own except where a call says so (texture attach,
 * stacked MIP bounds, the autotuners) and never falls back to the CPU.
 *
 * Errors.  Every function returns VR_OK (0) or a negative VR_ERR_* code;
 * vr_last_error() then gives a message (thread-local, valid until the next
 * failing call on that thread).
 *
 * Thread safety.  Distinct volumes may be used from distinct threads.  A
 * volume must not be modified (vr_set_transfer, vr_volume_upload,
 * vr_volume_destroy) while another thread uses it.
 */
#ifndef VR_H
#define VR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VR_OK 0
#define VR_ERR_ARG (-1)          /* invalid argument (null, size, alignment) */
#define VR_ERR_OOM (-2)          /* caller-provided buffer too small        */
#define VR_ERR_CUDA (-3)         /* a CUDA call or kernel launch failed      */
#define VR_ERR_TIMEOUT (-4)      /* a bounded device wait gave up            */
#define VR_ERR_UNSUPPORTED (-5)  /* feature not available on this device    */

#define VR_BRICK 32              /* bricks are 32 x 32 x 32 voxels           */
#define VR_MAX_LUT 256           /* largest transfer-function table          */

typedef enum { VR_F32 = 0, VR_F16 = 1, VR_I8 = 2 } vr_dtype;
typedef enum { VR_MIP = 0, VR_COMPOSITE = 1, VR_SUM = 2 } vr_mode;
typedef enum { VR_ORTHO = 0, VR_PERSP = 1 } vr_proj;

/* One camera, 64 bytes, lengths in voxel units (paper §3.1 item 3: the
 * camera is what maps each output pixel to a ray).  du and dv are the image
 * plane's per-pixel steps (for VR_PERSP at unit distance from the eye);
 * pixel rows run along dv.  `reserved` must be zero.                     */
typedef struct {
    int32_t proj;
    float eye[3];
    float fwd[3];
    float du[3];
    float dv[3];
    float reserved[3];
} vr_camera;

typedef struct vr_volume_s* vr_volume;

/* Device bytes a volume of the given dims (nx, ny, nz: x = RA fastest,
 * y = Dec, z = frequency channel slowest) and storage dtype occupies: the
 * voxels in 32^3 bricks (the paper's sub-cube partitioning, §3.1 process
 * item 1, at on-chip granularity), plus for VR_I8 two float tables of nz
 * entries.  Each dim must be in [2, 2^20] and the padded voxel count below
 * 2^40.                                                                    */
int vr_volume_bytes(const int64_t dims[3], int dtype, size_t* bytes_out);

/* Device bytes the library itself would allocate for a volume of these
 * dims and dtype, so a caller can budget memory before attaching anything
 * (paper abstract: data sets larger than GPU memory; §3.1 item 3's
 * trilinear fetch is what the texture storage serves):
 *   vr_texture_bytes     texture storage (vr_volume_attach_texture, or with
 *                        pair != 0 vr_volume_attach_pair_texture; FP16 /
 *                        int8 only): every layer's texels on the current
 *                        device's layered-texture layout, plus int8 decode
 *                        records.  VR_ERR_UNSUPPORTED beyond the device's
 *                        layered-texture limits or for FP32 pairs.
 *   vr_mip_bounds_bytes  MIP bounds of an FP32 volume with texture storage
 *                        (vr_volume_attach_mip_bounds): 8-bit codes of two
 *                        planes per 2-byte texel, nz + 1 cell slices
 *                        stacked as the texture, plus a 32-byte scale
 *                        record.  Filling them
 *                        also takes a stream-ordered scratch buffer of at
 *                        most 256 MiB, released on the stream.
 * The figures count the texels; the driver may round an allocation up to
 * its page size (2 MiB) and tile boundaries.  An attach that cannot get its
 * memory fails with VR_ERR_OOM and says how many bytes it asked for.      */
int vr_texture_bytes(const int64_t dims[3], int dtype, int pair, size_t* bytes_out);
int vr_mip_bounds_bytes(const int64_t dims[3], size_t* bytes_out);

/* Device bytes a volume holds now: *library_bytes the library's own
 * allocations (texture storage and MIP bounds, as the two calls above
 * count them), *caller_bytes the caller's buffers bound to it (the brick
 * buffer as passed to vr_volume_create -- 0 once dropped -- and the
 * empty-space masks).  Either pointer may be NULL.                         */
int vr_volume_device_bytes(vr_volume vol, size_t* library_bytes, size_t* caller_bytes);

/* Bind a caller-owned device buffer as a volume and, when src is not NULL,
 * pack the whole cube into it.
 *   dims         nx, ny, nz as above.
 *   dtype        storage type: VR_F32 (as given), VR_F16 (round to nearest
 *                even), VR_I8 (per frequency plane z: lo = min, hi = max,
 *                scale = (hi - lo)/254, offset = (hi + lo)/2, code =
 *                clamp(rint((v - offset)/scale), -127, 127); a constant
 *                plane gets scale 1 and code 0).  Decoding is
 *                code * scale + offset; a sample is the trilinear value
 *                of the decoded voxels (texture storage interpolates each
 *                plane's codes and decodes that: the same value up to
 *                FP32 rounding, as decoding is affine).
 *   src          float32 cube, linear, x fastest (nz*ny*nx values), or NULL
 *                to bind without data (fill later with vr_volume_upload).
 *   src_on_device 1: src is device memory.  0: src is page-locked host memory
 *                (e.g. cudaHostAlloc'ed or registered), read by the packing
 *                kernels directly; pageable host memory is rejected.
 *   brick_buf    device memory of at least vr_volume_bytes(), 256-byte
 *                aligned; owned by the caller, must outlive the volume.
 *   stream       cudaStream_t as void*; src may be released once the stream
 *                has passed this call.
 *   out          receives the handle (library-owned host memory; release
 *                with vr_volume_destroy).
 * The volume starts with a default transfer function (clip -inf, a grey
 * ramp over [0, 1], no early termination).                                 */
int vr_volume_create(const int64_t dims[3], int dtype, const float* src,
                     int src_on_device, void* brick_buf, size_t brick_bytes,
                     void* stream, vr_volume* out);

/* Pack planes [z0, z0 + nplanes) of the cube from a float32 source holding
 * exactly those planes (nplanes*ny*nx values, x fastest).  Lets a cube be
 * filled in slabs of frequency channels.  src_on_device and stream as in
 * vr_volume_create.  With texture storage the planes' slices of the texture
 * (and of the MIP bounds) are refreshed too: stream-ordered for an FP32
 * texture without stacked slices; otherwise through a surface, the call
 * then waiting for `stream`.                                               */
int vr_volume_upload(vr_volume vol, int64_t z0, int64_t nplanes, const float* src,
                     int src_on_device, void* stream);

/* Set the transfer function (paper §3.1 item 3, "pre-selected transfer
 * function"; abstract: low signal-to-noise emphasis -> the clip).
 *   rgba_lut     host memory, n entries of (r, g, b, alpha), alpha per unit
 *                voxel length in [0, 1]; copied, may be freed on return.
 *   n            2 .. VR_MAX_LUT.
 *   v_lo < v_hi  value domain the table spans (values outside clamp).
 *   clip         samples below clip are skipped (transparent).
 *   term_alpha   composite rays stop once A >= term_alpha (1 = only when
 *                fully opaque; values > 1 disable termination).
 * Applies to renders issued after the call returns.                        */
int vr_set_transfer(vr_volume vol, const float* rgba_lut, int n, float v_lo,
                     float v_hi, float clip, float term_alpha);

/* Render n_views images of w x h pixels (spec call; paper §3.1 item 3
 * and item 4: one image per view at the output resolution).
 *   cams         host array of n_views cameras; copied, may be freed on
 *                return.
 *   n_views, w, h  at least 1 each (VR_ERR_ARG for an empty image set).
 *   mode         VR_MIP / VR_COMPOSITE / VR_SUM.
 *   step         sample spacing in voxel lengths, > 0, and small enough
 *                that no ray takes 2^24 samples or more.
 *   out          device memory, 16-byte aligned for COMPOSITE (4-byte for
 *                MIP and SUM): view-major, then row py,
 *                then column px; 1 float per pixel (MIP, SUM) or 4 floats
 *                (COMPOSITE: premultiplied r, g, b, A).
 *   stream       cudaStream_t as void*.                                     */
int vr_render(vr_volume vol, const vr_camera* cams, int n_views, int w, int h,
              int mode, float step, float* out, void* stream);

/* As vr_render, and also adds to *d_samples (device memory, 8-byte aligned)
 * the number of samples evaluated: K per ray for MIP and SUM; for COMPOSITE
 * the samples up to and including the one that ended the ray.              */
int vr_render_counted(vr_volume vol, const vr_camera* cams, int n_views, int w,
                      int h, int mode, float step, float* out,
                      unsigned long long* d_samples, void* stream);

/* MIP in object order (paper §3.1 process items 1-5: the cube partitioned
 * into sub-cubes, each ray cast into an image, the images combined): the
 * cube is cut into sub-cubes of 32^3 cells; one thread block stages a
 * sub-cube's voxels from the bricks into shared memory once and renders,
 * for every view of the call (in launches of up to 64 views), the samples
 * of every ray that fall in it, combining the rays' partial maxima in `out`
 * with atomic maxima.  The same images and sample counts as vr_render's
 * MIP, bit for bit: each sample is taken by exactly one sub-cube and
 * computed with vr_render's arithmetic.  Reads the bricks (not the texture
 * storage; VR_ERR_UNSUPPORTED once they were dropped); `out` is first
 * filled with -inf.  mode must be VR_MIP (VR_ERR_ARG otherwise: the
 * composite needs each ray's samples in order).  d_samples may be NULL.
 * Other arguments as in vr_render.                                         */
int vr_render_object_order(vr_volume vol, const vr_camera* cams, int n_views, int w, int h,
                           int mode, float step, float* out, unsigned long long* d_samples,
                           void* stream);

/* Bytes of the volume's empty-space masks: 8 bytes per macrocell of
 * 4 x 4 x 4 cells, (nx/4 + 1) * (ny/4 + 1) * (nz/4 + 1) macrocells (integer
 * division; the gather coordinates 0 .. n of every axis, four per macrocell).
 * Host-only; no device work.                                                */
int vr_volume_mask_bytes(vr_volume vol, size_t* bytes_out);

/* Give the volume empty-space masks in the caller-owned device buffer `buf`
 * (16-byte aligned, at least vr_volume_mask_bytes bytes; the caller keeps it
 * alive while the volume renders).  COMPOSITE renders of a texture-stored
 * volume then skip the fetch and evaluation of samples whose cell cannot
 * reach the clip level (such samples are transparent: §3.1 item 3 with the
 * noise clip), with the warp's rays kept in step.  The masks depend on the
 * clip: they are built on the render's stream by the first COMPOSITE render
 * (or autotune) after this call or after a vr_volume_upload, and rebuilt
 * when vr_set_transfer lowers the clip below the level they were built for
 * (masks for a lower clip stay valid, only less tight, when the clip rises:
 * attach again to rebuild them tight).  Images and sample counts are identical to
 * those without masks; only the work differs.  MIP, SUM, brick-gather and
 * batched renders do not use them.  buf = NULL detaches.  No device work
 * here.  The paper describes no such structure.                            */
int vr_volume_attach_masks(vr_volume vol, void* buf, size_t bytes);

/* Build the attached masks now, for the current clip, from the bricks, on
 * `stream` (attached masks are otherwise built by the next composite render
 * that needs them).  For volumes whose brick buffer is about to hold other
 * data, such as part volumes sharing one buffer (a later build would read
 * whatever the buffer then holds).  vr_render_part uses a part's masks only
 * while they hold for its clip and never rebuilds them.  VR_ERR_UNSUPPORTED
 * without attached masks or after vr_volume_drop_bricks.                    */
int vr_volume_build_masks(vr_volume vol, void* stream);

/* Give the volume texture storage: a copy of the cube in one layered 2-D
 * texture, one 2-D slice per frequency plane, filled from the bricks on
 * `stream`.  A layered texture has at most 2048 layers: deeper cubes stack
 * 2^s slices per layer (the smallest s that fits), each with a copy of its
 * first and last row around it.  Renders then gather the 2 x 2 corners of a
 * cell per plane with the texture unit's four-texel gather (unfiltered
 * texels; the interpolation stays the kernel's own FP32 lerps).  This is the
 * one place the library allocates device memory: about
 * nx*ny*nz*sizeof(storage) bytes (for VR_I8 also 8 or 16 bytes per slice:
 * the planes' scales and offsets), owned by the volume and released by
 * vr_volume_detach_texture or vr_volume_destroy.  The call synchronises
 * `stream` (the fill must finish before its surface object is released).
 * Returns VR_ERR_UNSUPPORTED when nx or the stacked height exceeds the
 * device's layered texture size, VR_ERR_OOM when the allocation fails.      */
int vr_volume_attach_texture(vr_volume vol, void* stream);

/* Texture storage in pair format, for VR_F16 and VR_I8 volumes: each texel
 * packs a voxel with its neighbour in the next frequency plane (two binary16
 * values in 32 bits, or two int8 codes, each plus 128, in 16 bits), one 2-D slice per cell
 * plane (nz - 1 of them, stacked as in vr_volume_attach_texture), so one
 * four-texel gather returns all eight corners of a cell.  About twice the
 * bytes of vr_volume_attach_texture; replaces a plain texture storage if one
 * is attached.  Otherwise as vr_volume_attach_texture; VR_F32 volumes give
 * VR_ERR_UNSUPPORTED.                                                       */
int vr_volume_attach_pair_texture(vr_volume vol, void* stream);

/* Release the texture storage (renders fall back to gathering from the
 * bricks) and its MIP bounds.  The caller must make sure no render using it
 * is pending.                                                               */
int vr_volume_detach_texture(vr_volume vol);

/* MIP bounds for a VR_F32 volume with (plain) texture storage: a second
 * layered texture holding every voxel v as an 8-bit code c with L + c delta
 * >= v, on one scale for the whole cube (L its smallest finite voxel, 255
 * delta a little above its range), the two planes of a cell in one 2-byte
 * texel (cell slices, as the pair formats; about 2 bytes per voxel,
 * library-owned), so one four-texel gather returns the codes of all eight
 * corners of a sample's cell.  A MIP render (the maximum of the samples,
 * §3.1 process item 3) then marches the codes: their trilinear value bounds
 * the sample's value from above, and after allowing for the FP32 rounding
 * of both interpolations (2^-19 times the largest |voxel|, and the codes'
 * own rounding) a sample is read from the FP32 texture only when it could
 * raise the ray's running maximum.  The scale lives in device memory,
 * derived on the device when the bounds are attached and again when every
 * plane is uploaded.  MIP images and sample counts are those without bounds
 * bit for bit.  A cube the scale cannot cover (a +inf voxel, a range that
 * overflows, or a partial upload beyond the range) keeps its images but
 * evaluates every sample until the bounds are attached again.
 * MIP renders through vr_render_part use a part's bounds too; no effect on
 * COMPOSITE and SUM renders or on the batched launch.  Uploads refresh the
 * bounds with the texture.  VR_ERR_UNSUPPORTED for other storage types,
 * without texture storage, or after vr_volume_drop_bricks; VR_ERR_OOM when
 * an allocation fails.  The fill is queued on `stream` and the call returns
 * without waiting for it, except for cubes deep enough that the texture
 * stacks slices, where it waits for `stream`.  No counterpart in the
 * paper.                                                                    */
int vr_volume_attach_mip_bounds(vr_volume vol, void* stream);

/* Release the MIP bounds (MIP renders read the FP32 texture at every
 * sample again).  The caller must make sure no render using them is
 * pending.                                                                   */
int vr_volume_detach_mip_bounds(vr_volume vol);

/* Keep only the texture storage: after this call the volume renders from
 * its texture alone and never reads the brick buffer again, which the
 * caller may free once the work already queued on it has completed (the
 * call itself does no device work).  For volumes with texture storage
 * (an int8 texture carries its planes' scales and offsets).  Afterwards the
 * volume is read-only:
 * vr_volume_upload, vr_volume_detach_texture, vr_volume_attach_masks (other
 * than detaching) and a change of texture format return VR_ERR_UNSUPPORTED.
 * Empty-space masks already built stay, frozen at the clip level they were
 * built for: COMPOSITE renders at that clip or above use them, lower clips
 * render without them (nothing can rebuild them); masks never built are
 * detached.  No counterpart in the paper: it keeps cubes resident whose
 * bricks and texture would not both fit, e.g. several 32 GiB FP16 cubes.    */
int vr_volume_drop_bricks(vr_volume vol);

/* ---- cubes larger than the device: rendering part by part ---------------
 * The paper's pipeline partitions the cube into sub-cubes, renders each into
 * an image and composites the images (§3.1 items 1, 4, 5; abstract: data
 * larger than GPU memory).  Here a part is an ordinary volume holding planes
 * [z_first, z_first + nz) of the whole cube (with texture storage), and
 * vr_render_part continues images from the state they hold: each ray of the
 * whole cube takes, in order, its samples whose cell (floor of the sample
 * height) lies in [cell_lo, cell_hi), each sample computed exactly as the
 * one-pass vr_render computes it, so rendering every part in the rays' order
 * gives the one-pass images bit for bit.  Rays going up in z (sweep +1)
 * must see the parts in ascending order, rays going down (sweep -1) in
 * descending order: a caller renders the ascending sweep with sweep = +1
 * and the descending sweep with sweep = -1 (one of them is empty when every
 * ray of the views goes the same way; MIP needs no order but takes the same
 * calls).                                                                  */

/* Fill n_views images of w x h pixels with the empty state of `mode` (0 for
 * COMPOSITE and SUM, -inf for MIP) before the first vr_render_part.  out as
 * in vr_render.                                                            */
int vr_render_init(float* out, int n_views, int w, int h, int mode, void* stream);

/* Continue the images in `out` with the part's samples (see above).
 *   part         volume of planes [z_first, z_first + nz_part) of the cube,
 *                with texture storage; its transfer function is used.
 *   full_dims    the whole cube's nx, ny (equal to the part's), nz.
 *   cell_lo, cell_hi  cells [cell_lo, cell_hi) (the cell between planes c
 *                and c + 1 is cell c), within the part's planes:
 *                z_first <= cell_lo <= cell_hi <= z_first + nz_part - 1.
 *                cell_lo = 0 also takes positions a rounding error below
 *                plane 0, cell_hi = nz - 1 those above the top plane.  The
 *                parts' ranges must tile [0, nz - 1).
 *   sweep        +1: rays with dz >= 0; -1: rays with dz < 0; 0: every
 *                ray (a sub-cube's partial image, see
 *                vr_integrate_partials).
 *   out          images as left by vr_render_init or earlier parts.
 *   d_samples    optional count of evaluated samples (added to).
 * Other arguments as in vr_render.  COMPOSITE rays that terminated in an
 * earlier part are left as they are.                                       */
int vr_render_part(vr_volume part, const int64_t full_dims[3], int64_t z_first,
                   int64_t cell_lo, int64_t cell_hi, const vr_camera* cams, int n_views,
                   int w, int h, int mode, float step, int sweep, float* out,
                   unsigned long long* d_samples, void* stream);

/* Scene integration (paper §3.1 items 4, 5: each sub-cube rendered into its
 * own image, the images combined; read as the compositing operator applied
 * in visibility order).  Each sub-cube's partial image is its part's
 * vr_render_part with sweep 0 into images fresh from vr_render_init, so the
 * parts can be rendered in any order, or on different streams; this call
 * combines them, per pixel, in the order the pixel's ray meets them
 * (ascending z when its direction's height component is >= 0, computed as
 * vr_render computes it; descending otherwise):
 *   COMPOSITE  C += (1 - A) C_i, A += (1 - A) A_i  (premultiplied RGBA)
 *   MIP        the maximum;  SUM  the sum.
 * Without early termination (term_alpha > 1) the result equals the
 * one-pass image up to FP32 rounding (the operator is associative); with
 * it, each sub-cube stops at its own opacity, so a ray keeps, attenuated,
 * what lies behind an opaque sub-cube.
 *   partials     device memory, aligned as vr_render's `out`: n_parts image sets in
 *                sub-cube order (ascending z), each laid out as vr_render's
 *                `out` for n_views views of w x h (1 or 4 floats a pixel).
 *   cams         the n_views cameras the partial images were rendered with
 *                (host, copied).
 *   out          device memory, aligned as vr_render's `out`, one image set; it must not
 *                overlap `partials` (VR_ERR_ARG).
 * Asynchronous on `stream`; an HBM-bound kernel reading every partial image
 * once.  VR_ERR_ARG for null, misaligned or non-device pointers, n_parts <
 * 1, an empty image set, an unknown mode or a bad camera.                   */
int vr_integrate_partials(const float* partials, int n_parts, const vr_camera* cams,
                          int n_views, int w, int h, int mode, float* out, void* stream);

/* ---- many requests in one persistent launch ------------------------------
 * The paper's scheduler maps available tasks onto the computing resources
 * (Fig. 1 caption; §3.1 module 1).  Here the tasks are the ray tiles (256
 * rays each, in the shape vr_batch_autotune chose) of every request and the
 * resources are the SMs of one GPU.                                         */

#define VR_BATCH_MAX 64          /* requests per kernel launch (more are split) */

/* A transfer function given per request (same meaning as vr_set_transfer). */
typedef struct {
    const float* rgba_lut;       /* host, n x (r, g, b, alpha per unit length) */
    int32_t n;
    float v_lo, v_hi, clip, term_alpha;
} vr_transfer;

typedef struct {
    vr_volume vol;               /* texture storage is used when attached      */
    vr_camera cam;               /* one view                                   */
    int32_t w, h, mode;          /* image size; VR_MIP / VR_COMPOSITE / VR_SUM  */
    float step;
    float* out;                  /* device, aligned as vr_render's, one view   */
    const vr_transfer* tf;       /* host; NULL: the volume's transfer function */
    unsigned long long* samples; /* optional device counter (8-byte aligned):
                                    the evaluated samples are added to it      */
    unsigned int* done;          /* optional: device or mapped host word set to
                                    done_value once this request's image is
                                    complete (written after a system fence)    */
    unsigned int done_value;
    int32_t row0, rows;          /* rows > 0: render only rows [row0, row0 +
                                    rows) of the w x h image (the same rays,
                                    bit for bit), `out` holding just those rows
                                    (rows x w pixels); rows = 0 (and row0 = 0):
                                    the whole image.  Lets a caller split a
                                    large view over several launches.          */
} vr_request;

/* Bytes of device workspace vr_render_batch needs (work and tile counters). */
size_t vr_batch_workspace_bytes(void);

/* Render n requests -- any mix of volumes, storage types, resolutions,
 * modes and transfer functions -- with one persistent kernel launch per
 * VR_BATCH_MAX requests (also split when a launch would need more than 8
 * textured volumes or 2 distinct opacity-corrected tables; requests on
 * volumes with pair-texel texture storage, with plain texture storage and
 * without texture storage go to separate launches, in that order, each
 * kernel keeping the warps resident that its registers allow); n = 0
 * enqueues nothing and returns VR_OK.  Every request is
 * checked before anything is enqueued, so an argument error leaves the
 * stream untouched.  Each
 * block takes the next ray tile from a work counter in `workspace`
 * (caller-owned device memory of vr_batch_workspace_bytes(), 16-byte
 * aligned; zeroed on the stream by this call) and renders it with the same
 * per-ray arithmetic as vr_render, so every image equals the one vr_render
 * gives for the same request.  Requests, their tables and cameras are copied: the host arrays
 * may be reused on return.  Asynchronous on `stream`; the launches contain
 * no host synchronisation and can be captured into a CUDA graph (the
 * captured graph replays the same requests).                               */
int vr_render_batch(const vr_request* reqs, int n, void* workspace, size_t ws_bytes,
                    void* stream);

/* vr_render_batch for callers that cannot allocate device memory (no
 * counterpart in the paper: this is a deployment convenience).  Code that
 * must not allocate -- a fixed-budget real-time loop, a plugin handed no
 * allocator, a process that may not grow after start-up -- cannot supply
 * the workspace vr_render_batch asks for.  This call renders the same
 * requests the same way but keeps its work and tile counters in a fixed
 * array inside the library's device image (260 bytes on every GPU that
 * loads the library, held until the process exits).  It allocates no device
 * memory and calls nothing that does; on the host, the first batch call on
 * each thread (this one or vr_render_batch) makes that thread's launch
 * parameter block once, and later calls allocate nothing.
 *   n <= VR_BATCH_MAX; larger batches are rejected with VR_ERR_ARG (use
 *   vr_render_batch).  The first call in each CUDA context looks up the
 *   array's device address (cudaGetSymbolAddress) and keeps it for that
 *   context; make that first call before any stream capture.  A device reset
 *   ends the context, and the next call looks the address up again.  Each
 *   device (each context) has its own copy of the array, so calls on
 *   different devices are independent; calls on one device share it, and
 *   each launch zeroes it on `stream` before use, so two of these calls on
 *   the same device whose work overlaps on the GPU (different streams)
 *   race and must be ordered by the caller.                                  */
int vr_render_batch_noalloc(const vr_request* reqs, int n, void* stream);

/* Tile and ray-packet shapes of the batched launch (the batch autotuner's
 * search space): configuration cfg in [0, vr_batch_tune_count()) splits
 * every image into tiles of tile_x x tile_y rays (256, one block each) whose
 * warps hold packet_x x packet_y neighbouring rays.  Any output pointer may
 * be NULL.  Images do not depend on the shape.                             */
int vr_batch_tune_count(void);
int vr_batch_tune_describe(int cfg, int* tile_x, int* tile_y, int* packet_x, int* packet_y);

/* The shape every later vr_render_batch and vr_render_batch_noalloc call of
 * this process uses (initially 0; a process-wide setting, so callers on
 * several threads share it).  vr_get_batch_config returns it.              */
int vr_set_batch_config(int cfg);
int vr_get_batch_config(void);

/* Time every batch shape on these requests (arguments as vr_render_batch;
 * the images are written to the requests' outputs, each shape's run
 * overwriting the last) and keep the fastest as the process-wide shape.  A
 * tuning call, not a render call: it records events on `stream` and waits
 * for them, so it must not be captured into a CUDA graph.  n = 0 sets
 * *best_ms to -1 and changes nothing.                                        */
int vr_batch_autotune(const vr_request* reqs, int n, void* workspace, size_t ws_bytes,
                      void* stream, int* best_cfg, float* best_ms);

/* Launch shapes of the texture-gather kernel (the autotuner's search space):
 * configuration cfg in [0, vr_tune_count()) renders blocks of block_x x
 * block_y rays with warps holding packet_x x packet_y neighbouring rays, and
 * asks the compiler for registers that let min_blocks blocks share an SM.   */
int vr_tune_count(void);
int vr_tune_describe(int cfg, int* block_x, int* block_y, int* packet_x, int* packet_y,
                     int* min_blocks);

/* Time every launch shape on this render (same arguments as vr_render; the
 * images are written to `out`) and keep the fastest for `mode` on this
 * volume.  A tuning call, not a render call: it records events on `stream`
 * and waits for them, so it must not be captured into a CUDA graph.  Without
 * texture storage there is nothing to choose and *best_ms is set to -1.    */
int vr_autotune(vr_volume vol, const vr_camera* cams, int n_views, int w, int h, int mode,
                float step, float* out, void* stream, int* best_cfg, float* best_ms);

/* Use launch shape cfg for renders of `mode` on this volume (the default is
 * 0, or whatever vr_autotune chose last).                                    */
int vr_set_launch_config(vr_volume vol, int mode, int cfg);

/* Release the handle (not the caller's brick buffer).  The caller must make
 * sure no work using the volume is still pending on any stream.             */
int vr_volume_destroy(vr_volume vol);

/* Dimensions, dtype and device pointer of a volume (any pointer may be
 * NULL).                                                                     */
int vr_volume_info(vr_volume vol, int64_t dims[3], int* dtype, void** brick_buf);

/* The checked build (the library compiled with VR_DEBUG: libvr_debug.so,
 * no counterpart in the paper; a bounds checker built into the kernels,
 * standing in for an external memory checker): the texture-gather, part, batched, integration
 * and object-order kernels test every output index, brick address,
 * partial-image index, batched tile and staged sample they compute against
 * the buffer it addresses; a
 * failed test sets a bit and skips the access, never trapping.  This call
 * waits for the device, stores the bits recorded since the last clear in
 * *flags (1 output pixel outside the image set, 2 brick address outside the
 * brick buffer, 4 partial-image index outside the integration's input, 8 a
 * batched tile outside its request, 16 an object-order sample outside its
 * staged sub-cube, 0x80000000 the words could not be read)
 * and clears them when `clear` is non-zero.  VR_ERR_UNSUPPORTED (with *flags
 * = 0) in the regular build.                                                */
int vr_debug_status(unsigned* flags, int clear);

/* Message for the last failing call on this thread ("" if none).           */
const char* vr_last_error(void);

/* ABI version of this header: 2 (2 added vr_request's row band, making the
 * record 136 bytes).                                                        */
int vr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VR_H */
