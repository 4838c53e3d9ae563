// vr_api.cpp -- the C ABI of libvr (declared in include/vr.h): argument
// validation, volume handles, transfer-function preparation and launch
// planning.  No device memory is allocated here; all of it is the caller's.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "vr_internal.h"

namespace {

// An NVTX range around an entry point (named "vr_render" etc.), so a
// profiler's timeline shows the library's calls around their kernels; the
// header-only NVTX calls do nothing unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(VR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t align_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// Macrocells of the empty-space masks: every axis covers gather coordinates
// 0 .. n (cells -1 .. n - 1), four per macrocell.
size_t mask_macrocells(const vr::VolumeGeom& g)
{
    return (size_t)((g.nx >> vr::kMacroShift) + 1) * ((g.ny >> vr::kMacroShift) + 1) *
           ((g.nz >> vr::kMacroShift) + 1);
}

size_t elem_size(int dtype) { return dtype == VR_F32 ? 4 : dtype == VR_F16 ? 2 : 1; }

int check_dims(const int64_t dims[3], int dtype, vr::VolumeGeom* g)
{
    if (!dims) return fail(VR_ERR_ARG, "dims is NULL");
    if (dtype != VR_F32 && dtype != VR_F16 && dtype != VR_I8)
        return fail(VR_ERR_ARG, "unknown dtype %d", dtype);
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || dims[a] > (int64_t(1) << 20))
            return fail(VR_ERR_ARG, "dims[%d] = %lld outside [2, 2^20]", a, (long long)dims[a]);
    int64_t nb[3];
    for (int a = 0; a < 3; ++a) nb[a] = div_up(dims[a], vr::kBrick);
    const double voxels = (double)nb[0] * nb[1] * nb[2] * vr::kBrickVoxels;
    if (voxels >= std::ldexp(1.0, 40)) return fail(VR_ERR_ARG, "volume too large (>= 2^40 voxels)");
    g->nx = (int)dims[0];
    g->ny = (int)dims[1];
    g->nz = (int)dims[2];
    g->nbx = (int)nb[0];
    g->nby = (int)nb[1];
    g->nbz = (int)nb[2];
    return VR_OK;
}

// Is p device memory of the current device?  (Managed memory counts.)
bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = -1;
    cudaGetDevice(&dev);
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// Device-visible address of a page-locked host pointer, or nullptr.
const void* host_to_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost) return nullptr;
    return a.devicePointer;
}

// Images are written a pixel at a time: 16-byte stores of RGBA for
// COMPOSITE, 4-byte stores for MIP and SUM.
int out_alignment(int mode) { return mode == VR_COMPOSITE ? 16 : 4; }

bool finite3(const float v[3])
{
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

void default_transfer(vr::Volume* v)
{
    v->n_lut = 2;
    const float lut[2][4] = {{0, 0, 0, 0}, {1, 1, 1, 1}};
    std::memcpy(v->lut_raw, lut, sizeof lut);
    v->v_lo = 0.0f;
    v->v_hi = 1.0f;
    v->clip = -INFINITY;
    v->term_alpha = 2.0f;
    v->lut_valid = false;
}

// Opacity-corrected table for the given step: alpha' = 1 - (1 - alpha)^step
// (alpha is per unit voxel length), computed in double and rounded once.
void prepare_lut(vr::Volume* v, float step)
{
    if (v->lut_valid && v->lut_step == step) return;
    for (int i = 0; i < v->n_lut; ++i) {
        for (int c = 0; c < 3; ++c) v->lut_corr[i][c] = v->lut_raw[i][c];
        const double a = v->lut_raw[i][3];
        v->lut_corr[i][3] = (float)(1.0 - std::pow(1.0 - a, (double)step));
    }
    v->lut_step = step;
    v->lut_valid = true;
}

// Validate a render request and fill the launch parameters (all but the
// cameras and the output pointer, which are set per launch of <= 64 views).
int prepare(vr_volume vol, const vr_camera* cams, int n_views, int w, int h, int mode,
            float step, float* out, unsigned long long* d_samples, vr::MarchParams* p,
            vr::TexParams* tp)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    if (!cams) return fail(VR_ERR_ARG, "cams is NULL");
    if (n_views < 1) return fail(VR_ERR_ARG, "n_views = %d < 1", n_views);
    if (w < 1 || h < 1 || w > 65536 || h > 65536)
        return fail(VR_ERR_ARG, "image size %d x %d outside [1, 65536]", w, h);
    if (mode != VR_MIP && mode != VR_COMPOSITE && mode != VR_SUM)
        return fail(VR_ERR_ARG, "unknown mode %d", mode);
    if (!(step > 0.0f) || !std::isfinite(step)) return fail(VR_ERR_ARG, "step must be > 0");
    const double hx = v->g.nx - 1.0, hy = v->g.ny - 1.0, hz = v->g.nz - 1.0;
    const double diag = std::sqrt(hx * hx + hy * hy + hz * hz);
    if (diag / step + 2.0 >= 16777216.0)
        return fail(VR_ERR_ARG, "step %g too small: a ray could take 2^24 samples", (double)step);
    if (!out) return fail(VR_ERR_ARG, "out is NULL");
    if (reinterpret_cast<uintptr_t>(out) % out_alignment(mode) != 0)
        return fail(VR_ERR_ARG, "out must be %d-byte aligned", out_alignment(mode));
    if (!is_device_ptr(out)) return fail(VR_ERR_ARG, "out is not device memory of this device");
    if (d_samples) {
        if (reinterpret_cast<uintptr_t>(d_samples) % 8 != 0)
            return fail(VR_ERR_ARG, "d_samples must be 8-byte aligned");
        if (!is_device_ptr(d_samples)) return fail(VR_ERR_ARG, "d_samples is not device memory");
    }
    for (int i = 0; i < n_views; ++i) {
        const vr_camera& c = cams[i];
        if (c.proj != VR_ORTHO && c.proj != VR_PERSP)
            return fail(VR_ERR_ARG, "camera %d: unknown projection %d", i, c.proj);
        if (!finite3(c.eye) || !finite3(c.fwd) || !finite3(c.du) || !finite3(c.dv))
            return fail(VR_ERR_ARG, "camera %d: non-finite parameters", i);
        if (c.fwd[0] == 0.0f && c.fwd[1] == 0.0f && c.fwd[2] == 0.0f)
            return fail(VR_ERR_ARG, "camera %d: zero forward vector", i);
    }

    std::memset(p, 0, sizeof *p);
    p->bricks = v->bricks;
    p->scale = v->scale;
    p->offset = v->offset;
    p->g = v->g;
    p->hix = (float)hx;
    p->hiy = (float)hy;
    p->hiz = (float)hz;
    p->w = w;
    p->h = h;
    p->step = step;
    p->clip = v->clip;
    p->term_alpha = v->term_alpha;
    p->v_lo = v->v_lo;
    p->lut_scale = (float)((v->n_lut - 1) / ((double)v->v_hi - (double)v->v_lo));
    p->lut_max = (float)(v->n_lut - 1);
    p->n_lut = v->n_lut;
    p->samples = d_samples;
    if (mode == VR_COMPOSITE) {
        prepare_lut(v, step);
        for (int i = 0; i < v->n_lut; ++i)
            p->lut[i] = make_float4(v->lut_corr[i][0], v->lut_corr[i][1], v->lut_corr[i][2],
                                    v->lut_corr[i][3]);
    }
    std::memset(tp, 0, sizeof *tp);
    tp->tex = v->tex;
    tp->stack_shift = v->stack_shift;
    tp->stack_pitch = v->stack_pitch;
    tp->dec = v->dec;
    tp->k_max = (int)(diag / step) + 2;
    tp->bound = v->bound_tex;
    tp->bound_scale = v->bound_scale;
    p->mask = v->mask;
    p->mnx = v->mnx;
    p->mny = v->mny;
    p->mlast = v->mask ? v->mnx * v->mny * v->mnz - 1 : 0;
    return VR_OK;
}

// Composite renders with empty-space masks need masks built for a clip level
// at or below the volume's clip (a cell that can reach the clip can reach
// any lower one, so masks for a lower clip are conservative): rebuild them
// (on the render's stream) when the clip has dropped below it.  A volume
// whose bricks were dropped keeps the masks built before, frozen: a clip
// below their level renders without them (p->mask cleared).
int ensure_masks(vr::Volume* v, int mode, cudaStream_t s, vr::MarchParams* p)
{
    if (!v->mask || mode != VR_COMPOSITE) return VR_OK;
    if (!std::isnan(v->mask_clip) && !(v->clip < v->mask_clip)) return VR_OK;
    if (v->texture_only) {
        p->mask = nullptr;
        return VR_OK;
    }
    cudaError_t e = vr::launch_masks(*v, v->clip, s);
    if (e != cudaSuccess) return cuda_fail(e, "mask launch");
    v->mask_clip = v->clip;
    return VR_OK;
}

// Launch the views in groups of at most kMaxViewsPerLaunch (cameras travel
// in the kernel parameters).  cfg: texture-kernel shape.
int launch_views(vr::Volume* v, vr::MarchParams& p, const vr::TexParams& tp, int mode, int cfg,
                 const vr_camera* cams, int n_views, float* out, cudaStream_t s)
{
    const size_t per_view = (size_t)p.w * p.h * (mode == VR_COMPOSITE ? 4 : 1);
    for (int v0 = 0; v0 < n_views; v0 += vr::kMaxViewsPerLaunch) {
        const int nv = std::min(vr::kMaxViewsPerLaunch, n_views - v0);
        p.n_views = nv;
        std::memcpy(p.cams, cams + v0, sizeof(vr_camera) * nv);
        p.out = out + per_view * v0;
        cudaError_t e = v->has_tex ? vr::launch_tex(p, tp, v->tex_format, mode, cfg, s)
                                        : vr::launch_march(p, v->dtype, mode, s);
        if (e != cudaSuccess) return cuda_fail(e, "march launch");
    }
    return VR_OK;
}

int render_impl(vr_volume vol, const vr_camera* cams, int n_views, int w, int h, int mode,
                float step, float* out, unsigned long long* d_samples, void* stream)
{
    vr::MarchParams p;
    vr::TexParams tp;
    int rc = prepare(vol, cams, n_views, w, h, mode, step, out, d_samples, &p, &tp);
    if (rc) return rc;
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    rc = ensure_masks(v, mode, static_cast<cudaStream_t>(stream), &p);
    if (rc) return rc;
    return launch_views(v, p, tp, mode, v->cfg[mode], cams, n_views, out,
                        static_cast<cudaStream_t>(stream));
}

// Every argument check of one request (the view as vr_render checks it, the
// completion word, the request's own transfer function).
int check_request(const vr_request& rq, int index)
{
    if (!rq.vol) return fail(VR_ERR_ARG, "request %d: volume is NULL", index);
    vr::MarchParams mp;
    vr::TexParams tp;
    int rc = prepare(rq.vol, &rq.cam, 1, rq.w, rq.h, rq.mode, rq.step, rq.out, rq.samples, &mp,
                     &tp);
    if (rc) return rc;
    if (rq.done && reinterpret_cast<uintptr_t>(rq.done) % 4 != 0)
        return fail(VR_ERR_ARG, "request %d: done must be 4-byte aligned", index);
    if (rq.rows < 0 || rq.row0 < 0 || (rq.rows == 0 && rq.row0 != 0) ||
        (int64_t)rq.row0 + rq.rows > rq.h)
        return fail(VR_ERR_ARG, "request %d: row band [%d, %d + %d) outside the %d rows", index,
                    rq.row0, rq.row0, rq.rows, rq.h);
    if (rq.tf) {
        const vr_transfer& t = *rq.tf;
        if (!t.rgba_lut || t.n < 2 || t.n > VR_MAX_LUT)
            return fail(VR_ERR_ARG, "request %d: bad transfer table", index);
        if (!std::isfinite(t.v_lo) || !std::isfinite(t.v_hi) || !(t.v_lo < t.v_hi) ||
            std::isnan(t.clip) || std::isnan(t.term_alpha))
            return fail(VR_ERR_ARG, "request %d: bad transfer domain", index);
        for (int i = 0; i < 4 * t.n; ++i)
            if (!std::isfinite(t.rgba_lut[i]) || ((i & 3) == 3 && (t.rgba_lut[i] < 0.0f ||
                                                                   t.rgba_lut[i] > 1.0f)))
                return fail(VR_ERR_ARG, "request %d: bad transfer table entry", index);
    }
    return VR_OK;
}

// Fill the kernel record of one (checked) request; tables and textured
// volumes are looked up in (or added to) the launch's slots.  Returns VR_OK
// or 1 when the launch has no free slot left (start a new launch).
int batch_request(const vr_request& rq, vr::BatchParams* B, int* n_tex, vr::Volume** tex_vols,
                  int* n_lut, float* lut_steps, int* lut_ns, int cfg)
{
    vr::Volume* v = reinterpret_cast<vr::Volume*>(rq.vol);
    vr::MarchParams mp;
    vr::TexParams tp;
    prepare(rq.vol, &rq.cam, 1, rq.w, rq.h, rq.mode, rq.step, rq.out, rq.samples, &mp, &tp);
    vr::BatchReq& q = B->req[B->n];
    std::memset(&q, 0, sizeof q);
    // transfer function: the request's own or the volume's
    const float* raw = &v->lut_raw[0][0];
    int nl = v->n_lut;
    float v_lo = v->v_lo, v_hi = v->v_hi, clip = v->clip, ta = v->term_alpha;
    if (rq.tf) {
        const vr_transfer& t = *rq.tf;
        raw = t.rgba_lut;
        nl = t.n;
        v_lo = t.v_lo;
        v_hi = t.v_hi;
        clip = t.clip;
        ta = t.term_alpha;
    }
    int lut_slot = 0;
    if (rq.mode == VR_COMPOSITE) {
        // opacity-corrected table for this step, shared with an identical one
        float4 corr[VR_MAX_LUT];
        for (int i = 0; i < nl; ++i) {
            const double a = raw[4 * i + 3];
            corr[i] = make_float4(raw[4 * i], raw[4 * i + 1], raw[4 * i + 2],
                                  (float)(1.0 - std::pow(1.0 - a, (double)rq.step)));
        }
        lut_slot = -1;
        for (int i = 0; i < *n_lut; ++i)
            if (lut_ns[i] == nl && std::memcmp(B->lut[i], corr, sizeof(float4) * nl) == 0)
                lut_slot = i;
        if (lut_slot < 0) {
            if (*n_lut == vr::kMaxBatchLut) return 1;
            lut_slot = (*n_lut)++;
            std::memcpy(B->lut[lut_slot], corr, sizeof(float4) * nl);
            lut_ns[lut_slot] = nl;
            lut_steps[lut_slot] = rq.step;
        }
    }
    int tex_slot = -1;
    if (v->has_tex) {
        for (int i = 0; i < *n_tex; ++i)
            if (tex_vols[i] == v) tex_slot = i;
        if (tex_slot < 0) {
            if (*n_tex == vr::kMaxBatchTex) return 1;
            tex_slot = (*n_tex)++;
            tex_vols[tex_slot] = v;
            vr::BatchTex& T = B->tex[tex_slot];
            std::memset(&T, 0, sizeof T);
            T.tex = v->tex;
            T.stack_shift = v->stack_shift;
            T.stack_pitch = v->stack_pitch;
            T.format = v->tex_format;
            T.dec = v->dec;
        }
    }
    q.cam = rq.cam;
    q.out = rq.out;
    q.bricks = v->bricks;
    q.scale = v->scale;
    q.offset = v->offset;
    q.samples = rq.samples;
    q.done = rq.done;
    q.done_value = rq.done_value;
    q.mask = nullptr;      // the batched kernel marches every sample
    q.g = v->g;
    q.hix = mp.hix;
    q.hiy = mp.hiy;
    q.hiz = mp.hiz;
    q.step = rq.step;
    q.clip = clip;
    q.term_alpha = ta;
    q.v_lo = v_lo;
    q.lut_scale = (float)((nl - 1) / ((double)v_hi - (double)v_lo));
    q.lut_max = (float)(nl - 1);
    q.n_lut = nl;
    q.k_max = tp.k_max;
    q.w = rq.w;
    q.h = rq.h;
    q.mode = rq.mode;
    q.dtype = v->dtype;
    q.tex_slot = tex_slot;
    q.lut_slot = lut_slot;
    // the rows this request renders: a band of the image, or all of it
    q.row0 = rq.rows > 0 ? rq.row0 : 0;
    q.row_end = rq.rows > 0 ? rq.row0 + rq.rows : rq.h;
    const vr::BatchShape& S = vr::kBatchShapes[cfg];
    q.tiles_x = (rq.w + S.tx - 1) / S.tx;
    q.n_tiles = q.tiles_x * ((q.row_end - q.row0 + S.ty - 1) / S.ty);
    q.first_item = B->total_items;
    B->total_items += q.n_tiles;
    B->n++;
    return VR_OK;
}

// A launch holds requests of one class (pair texels, plain texels, bricks),
// so that each kernel instance compiles one fetch path and keeps the warps
// its registers allow: the classes go in that order, each split into
// launches as its slots fill.
int batch_class(const vr_request& r)
{
    const vr::Volume* v = reinterpret_cast<const vr::Volume*>(r.vol);
    if (!v || !v->has_tex) return vr::kBatchBricks;
    const bool pair = v->tex_format == vr::kF16Pair || v->tex_format == vr::kI8Pair;
    return pair ? vr::kBatchTexPair : vr::kBatchTex;
}

// Tile and ray-packet shape of the batched launches (process-wide; set by
// vr_set_batch_config or vr_batch_autotune).
std::atomic<int> g_batch_cfg{0};

int batch_impl(const vr_request* reqs, int n, unsigned* ws, cudaStream_t s, int cfg)
{
    // persistent grid: as many blocks as fit on the current device at once
    // (cached per device, class and shape)
    constexpr int kDevices = 64;
    static std::atomic<int> grid[kDevices][vr::kNumBatchClasses][vr::kNumBatchShapes];
    int dev = 0;
    cudaGetDevice(&dev);
    int g[vr::kNumBatchClasses];
    for (int c = 0; c < vr::kNumBatchClasses; ++c) {
        g[c] = dev >= 0 && dev < kDevices ? grid[dev][c][cfg].load() : 0;
        if (g[c] == 0) {
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (sms < 1) sms = 1;
            g[c] = sms * vr::batch_blocks_per_sm(c, cfg);
            if (dev >= 0 && dev < kDevices) grid[dev][c][cfg].store(g[c]);
        }
    }
    // every request is checked before anything is enqueued, so an argument
    // error leaves the stream untouched
    for (int i = 0; i < n; ++i) {
        const int rc = check_request(reqs[i], i);
        if (rc) return rc;
    }
    // the launch parameter block (about 25 KB, copied into each launch):
    // one per thread, made at the thread's first batch call, so later calls
    // allocate no host memory either
    static thread_local std::unique_ptr<vr::BatchParams> tls_params;
    if (!tls_params) {
        tls_params.reset(new (std::nothrow) vr::BatchParams);
        if (!tls_params) return fail(VR_ERR_OOM, "out of host memory");
    }
    vr::BatchParams* B = tls_params.get();
    int rc = VR_OK;
    const int order[vr::kNumBatchClasses] = {vr::kBatchTexPair, vr::kBatchTex,
                                             vr::kBatchBricks};
    for (int oi = 0; oi < vr::kNumBatchClasses && rc == VR_OK; ++oi) {
        const int cls = order[oi];
        int i = 0;
        while (rc == VR_OK) {
            while (i < n && batch_class(reqs[i]) != cls) ++i;    // other classes
            if (i >= n) break;
            B->n = 0;
            B->total_items = 0;
            int n_tex = 0, n_lut = 0;
            vr::Volume* tex_vols[vr::kMaxBatchTex];
            float lut_steps[vr::kMaxBatchLut];
            int lut_ns[vr::kMaxBatchLut];
            while (i < n && B->n < vr::kMaxBatch) {
                if (batch_class(reqs[i]) != cls) {
                    ++i;
                    continue;
                }
                const int r = batch_request(reqs[i], B, &n_tex, tex_vols, &n_lut, lut_steps,
                                            lut_ns, cfg);
                if (r == 1) break;       // slots full: launch what we have
                ++i;
            }
            if (rc == VR_OK && B->n > 0) {
                cudaError_t e = vr::launch_batch(*B, ws, g[cls], cls, cfg, s);
                if (e != cudaSuccess) rc = cuda_fail(e, "batch launch");
            }
        }
    }
    return rc;
}

void release_bounds(vr::Volume* v)
{
    if (v->bound_tex) cudaDestroyTextureObject(v->bound_tex);
    if (v->bound_array) cudaFreeArray(v->bound_array);
    if (v->bound_scale) cudaFree(v->bound_scale);
    v->bound_tex = 0;
    v->bound_array = nullptr;
    v->bound_scale = nullptr;
}

// MIP-bound cell slices holding planes [z0, z1): slice s packs planes s - 1
// and s (clamped), so plane z is in slices z and z + 1.
int fill_bound_planes(vr::Volume* v, int64_t z0, int64_t z1, cudaStream_t s);

// Fill MIP-bound slices [s0, s1) with the codes of the volume's bound scale
// (a voxel the scale does not cover turns skipping off, see BoundScale).
// An unstacked bound texture is written linearly to a stream-ordered scratch
// buffer and copied into the array, chunk by chunk, with no wait; a stacked
// one through a surface, the stream waited for before the surface object is
// destroyed.
int fill_bound_slices(vr::Volume* v, int64_t s0, int64_t s1, cudaStream_t s)
{
    if (s0 >= s1) return VR_OK;
    const int nx = v->g.nx, ny = v->g.ny;
    if (v->stack_shift == 0) {
        const size_t slice = (size_t)nx * ny * sizeof(unsigned short);
        const int64_t chunk =
            std::max<int64_t>(1, std::min<int64_t>(s1 - s0, (int64_t)((256u << 20) / slice)));
        unsigned short* buf = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), chunk * slice, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(VR_ERR_OOM, "MIP bound scratch: %s", cudaGetErrorString(e));
        }
        for (int64_t c0 = s0; c0 < s1 && e == cudaSuccess; c0 += chunk) {
            const int64_t c1 = std::min(s1, c0 + chunk);
            e = vr::fill_bounds_linear(*v, buf, (int)c0, (int)c1, s);
            if (e == cudaSuccess) {
                cudaMemcpy3DParms p;
                std::memset(&p, 0, sizeof p);
                p.srcPtr = make_cudaPitchedPtr(buf, (size_t)nx * sizeof(unsigned short), nx, ny);
                p.dstArray = v->bound_array;
                p.dstPos = make_cudaPos(0, 0, (size_t)c0);
                p.extent = make_cudaExtent(nx, ny, (size_t)(c1 - c0));
                p.kind = cudaMemcpyDeviceToDevice;
                e = cudaMemcpy3DAsync(&p, s);
            }
        }
        const cudaError_t e2 = cudaFreeAsync(buf, s);
        if (e != cudaSuccess) return cuda_fail(e, "bound fill");
        if (e2 != cudaSuccess) return cuda_fail(e2, "bound scratch");
        return VR_OK;
    }
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = v->bound_array;
    cudaSurfaceObject_t surf = 0;
    cudaError_t e = cudaCreateSurfaceObject(&surf, &rd);
    if (e != cudaSuccess) return cuda_fail(e, "surface object");
    e = vr::fill_bounds(*v, surf, (int)s0, (int)s1, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);   // before the surface object goes
    cudaDestroySurfaceObject(surf);
    if (e != cudaSuccess) return cuda_fail(e, "bound fill");
    if (e2 != cudaSuccess) return cuda_fail(e2, "bound fill");
    return VR_OK;
}

int fill_bound_planes(vr::Volume* v, int64_t z0, int64_t z1, cudaStream_t s)
{
    // new contents for every plane (a part volume taking its next part): the
    // scale is derived again from them
    if (z0 == 0 && z1 >= v->g.nz) {
        const cudaError_t e = vr::bound_scale(*v, s);
        if (e != cudaSuccess) return cuda_fail(e, "MIP bound scale");
    }
    return fill_bound_slices(v, z0, std::min<int64_t>(z1, v->g.nz) + 1, s);
}

void release_texture(vr::Volume* v)
{
    release_bounds(v);
    if (v->tex) cudaDestroyTextureObject(v->tex);
    if (v->array) cudaFreeArray(v->array);
    if (v->dec) cudaFree(v->dec);
    v->tex = 0;
    v->array = nullptr;
    v->dec = nullptr;
    v->has_tex = false;
}

// Copy planes [z0, z1) of the bricks into the texture (for pair formats: the
// cell planes whose texels include one of those planes).
int refresh_texture(vr::Volume* v, int64_t z0, int64_t z1, cudaStream_t s)
{
    // slices holding planes [z0, z1): plain slice s holds plane s - 1 (slices
    // 0 and nz + 1 repeat the edge planes); pair slice s holds planes s - 1
    // and s (clamped)
    const bool pair = v->tex_format == vr::kF16Pair || v->tex_format == vr::kI8Pair;
    const int64_t last = pair ? v->g.nz : v->g.nz + 1;
    int64_t s0 = z0 == 0 ? 0 : z0 + (pair ? 0 : 1);
    int64_t s1 = z1 == v->g.nz ? last + 1 : z1 + 1;
    if (s0 >= s1) return VR_OK;
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = v->array;
    cudaSurfaceObject_t surf = 0;
    cudaError_t e = cudaCreateSurfaceObject(&surf, &rd);
    if (e != cudaSuccess) return cuda_fail(e, "surface object");
    e = vr::fill_texture(*v, surf, (int)s0, (int)s1, s);
    if (e == cudaSuccess && v->dec) e = vr::fill_decode_records(*v, s);   // planes rescaled
    // the surface object may only be destroyed after the fill ran: wait
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaDestroySurfaceObject(surf);
    if (e != cudaSuccess) return cuda_fail(e, "texture fill");
    if (e2 != cudaSuccess) return cuda_fail(e2, "texture fill");
    if (v->bound_array) return fill_bound_planes(v, z0, z1, s);
    return VR_OK;
}

// FP32 texture storage without stacked slices holds the planes exactly as
// given: the uploaded planes [z0, z0 + n) are copied into their slices
// (slice z + 1), and the edge planes also into slices 0 and nz + 1 when the
// upload includes them; stream-ordered, like the fill it replaces.
int copy_texture_planes(vr::Volume* v, int64_t z0, int64_t n, const float* src, cudaStream_t s)
{
    const int nx = v->g.nx, ny = v->g.ny, nz = v->g.nz;
    auto copy = [&](int64_t plane, int64_t slice, int64_t depth) {
        cudaMemcpy3DParms p;
        std::memset(&p, 0, sizeof p);
        p.srcPtr = make_cudaPitchedPtr(const_cast<float*>(src), (size_t)nx * sizeof(float), nx, ny);
        p.srcPos = make_cudaPos(0, 0, (size_t)(plane - z0));
        p.dstArray = v->array;
        p.dstPos = make_cudaPos(0, 0, (size_t)slice);
        p.extent = make_cudaExtent(nx, ny, (size_t)depth);
        p.kind = cudaMemcpyDefault;
        return cudaMemcpy3DAsync(&p, s);
    };
    cudaError_t e = copy(z0, z0 + 1, n);
    if (e == cudaSuccess && z0 == 0) e = copy(0, 0, 1);
    if (e == cudaSuccess && z0 + n == nz) e = copy(nz - 1, nz + 1, 1);
    if (e != cudaSuccess) return cuda_fail(e, "texture copy");
    if (v->bound_array) return fill_bound_planes(v, z0, z0 + n, s);
    return VR_OK;
}

// Layered-texture layout of a cube on the current device: slices are planes
// (plain formats, nz + 2 with the edge planes repeated) or cells (pair, nz +
// 1), stacked 2^shift per layer (each with a copy of its edge rows) when they
// outnumber the layers.  Returns VR_OK or VR_ERR_UNSUPPORTED (beyond the
// device's layered-texture limits).
struct TexLayout {
    int slices, shift, pitch, layers;
};

int texture_layout(const vr::VolumeGeom& g, bool pair, TexLayout* L)
{
    int dev = 0;
    cudaGetDevice(&dev);
    int maxw = 0, maxh = 0, maxl = 0;
    cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture2DLayeredWidth, dev);
    cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxTexture2DLayeredHeight, dev);
    cudaDeviceGetAttribute(&maxl, cudaDevAttrMaxTexture2DLayeredLayers, dev);
    cudaGetLastError();
    maxl = std::min(maxl, vr::kMaxLayers);
    if (maxl < 1) maxl = vr::kMaxLayers;      // no device: the sm_103 limits
    if (maxw < 1) maxw = 32768;
    if (maxh < 1) maxh = 32768;
    L->slices = pair ? g.nz + 1 : g.nz + 2;
    L->shift = 0;
    while (((L->slices + (1 << L->shift) - 1) >> L->shift) > maxl) ++L->shift;
    L->pitch = L->shift > 0 ? g.ny + 2 : g.ny;
    L->layers = (L->slices + (1 << L->shift) - 1) >> L->shift;
    if (g.nx > maxw || (int64_t)L->pitch << L->shift > maxh)
        return fail(VR_ERR_UNSUPPORTED, "cube %d x %d x %d exceeds the layered texture limits",
                    g.nx, g.ny, g.nz);
    return VR_OK;
}

size_t texel_bytes(int format)
{
    switch (format) {
    case VR_F32: return 4;
    case VR_F16: return 2;
    case VR_I8: return 1;
    case vr::kF16Pair: return 4;
    default: return 2;            // kI8Pair
    }
}

// Device bytes of the texture storage (texels of every layer, plus the int8
// decode records) and of the MIP bounds (8-bit code pairs in cell slices,
// plus the scale record).
size_t texture_bytes(const vr::VolumeGeom& g, int format, const TexLayout& L)
{
    const size_t texels = (size_t)g.nx * ((size_t)L.pitch << L.shift) * L.layers;
    const bool pair = format == vr::kF16Pair || format == vr::kI8Pair;
    size_t dec = 0;
    if (format == VR_I8 || format == vr::kI8Pair) dec = (size_t)L.slices * (pair ? 16 : 8);
    return texels * texel_bytes(format) + dec;
}

// L: the layout of the bound texture's nz + 1 cell slices (see attach_bounds).
size_t bounds_bytes(const vr::VolumeGeom& g, const TexLayout& L)
{
    return (size_t)g.nx * ((size_t)L.pitch << L.shift) * L.layers * 2 + sizeof(vr::BoundScale);
}

// The bound texture's layout: the texture's stacking over nz + 1 cell slices.
TexLayout bound_layout(const vr::VolumeGeom& g, int shift, int pitch)
{
    const int slices = g.nz + 1;
    return TexLayout{slices, shift, pitch, (slices + (1 << shift) - 1) >> shift};
}

int attach_bounds(vr::Volume* v, cudaStream_t s)
{
    if (v->dtype != VR_F32)
        return fail(VR_ERR_UNSUPPORTED, "MIP bounds are for FP32 storage");
    if (!v->has_tex || v->tex_format != VR_F32)
        return fail(VR_ERR_UNSUPPORTED, "MIP bounds need texture storage (attach it first)");
    if (v->bound_array) return VR_OK;
    if (v->texture_only)
        return fail(VR_ERR_UNSUPPORTED, "the volume's bricks were dropped: no new bounds");
    // cell slices (the 8-bit codes of two planes per 16-bit texel, as the pair
    // formats) with the texture's stacking (vr_ray.cuh)
    const TexLayout L = bound_layout(v->g, v->stack_shift, v->stack_pitch);
    cudaChannelFormatDesc desc = cudaCreateChannelDesc<unsigned short>();
    cudaError_t e = cudaMalloc3DArray(
        &v->bound_array, &desc,
        make_cudaExtent(v->g.nx, (size_t)v->stack_pitch << v->stack_shift, L.layers),
        cudaArrayLayered | cudaArraySurfaceLoadStore);
    if (e != cudaSuccess) {
        cudaGetLastError();
        v->bound_array = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA,
                    "MIP bound storage of %zu bytes: %s", bounds_bytes(v->g, L),
                    cudaGetErrorString(e));
    }
    e = cudaMalloc(reinterpret_cast<void**>(&v->bound_scale), sizeof(vr::BoundScale));
    if (e != cudaSuccess) {
        cudaGetLastError();
        v->bound_scale = nullptr;
        release_bounds(v);
        return fail(VR_ERR_OOM, "MIP bound scale: %s", cudaGetErrorString(e));
    }
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = v->bound_array;
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof td);
    td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    e = cudaCreateTextureObject(&v->bound_tex, &rd, &td, nullptr);
    if (e != cudaSuccess) {
        v->bound_tex = 0;
        release_bounds(v);
        return cuda_fail(e, "MIP bound texture object");
    }
    e = vr::bound_scale(*v, s);
    if (e != cudaSuccess) {
        release_bounds(v);
        return cuda_fail(e, "MIP bound scale");
    }
    int rc = fill_bound_slices(v, 0, L.slices, s);
    if (rc) release_bounds(v);
    return rc;
}

int attach_texture(vr_volume vol, bool pair, void* stream)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    if (pair && v->dtype == VR_F32)
        return fail(VR_ERR_UNSUPPORTED, "pair textures hold FP16 or int8 storage only");
    const int format = pair ? (v->dtype == VR_F16 ? vr::kF16Pair : vr::kI8Pair) : v->dtype;
    if (v->texture_only) {
        if (v->tex_format == format) return VR_OK;
        return fail(VR_ERR_UNSUPPORTED, "the volume's bricks were dropped: no new texture");
    }
    if (v->has_tex) {
        if (v->tex_format == format) return VR_OK;
        release_texture(v);
    }
    TexLayout L;
    const int lrc = texture_layout(v->g, pair, &L);
    if (lrc) return lrc;
    const int slices = L.slices, shift = L.shift, pitch = L.pitch;
    cudaChannelFormatDesc desc = format == VR_F32    ? cudaCreateChannelDesc<float>()
                                 : format == VR_F16   ? cudaCreateChannelDescHalf()
                                 : format == VR_I8    ? cudaCreateChannelDesc<signed char>()
                                 : format == vr::kF16Pair ? cudaCreateChannelDesc<unsigned int>()
                                                          : cudaCreateChannelDesc<unsigned short>();
    cudaArray_t arr = nullptr;
    cudaError_t e = cudaMalloc3DArray(
        &arr, &desc,
        make_cudaExtent(v->g.nx, (size_t)pitch << shift, (slices + (1 << shift) - 1) >> shift),
        cudaArrayLayered | cudaArraySurfaceLoadStore);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA,
                    "texture storage of %zu bytes: %s", texture_bytes(v->g, format, L),
                    cudaGetErrorString(e));
    }
    v->array = arr;
    v->has_tex = true;
    v->tex_format = format;
    v->stack_shift = shift;
    v->stack_pitch = pitch;
    if (v->dtype == VR_I8) {
        // per-slice decode records (float2 plain, float4 pair)
        e = cudaMalloc(&v->dec, (size_t)slices * (pair ? 16 : 8));
        if (e != cudaSuccess) {
            cudaGetLastError();
            v->dec = nullptr;
            release_texture(v);
            return fail(VR_ERR_OOM, "texture decode records: %s", cudaGetErrorString(e));
        }
    }
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = arr;
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof td);
    td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    e = cudaCreateTextureObject(&v->tex, &rd, &td, nullptr);
    if (e != cudaSuccess) {
        release_texture(v);
        return cuda_fail(e, "texture object");
    }
    int rc = refresh_texture(v, 0, v->g.nz, static_cast<cudaStream_t>(stream));
    if (rc) release_texture(v);
    return rc;
}

}  // namespace

namespace vr {

// Entry points for the allocation-free batch call (vr_noalloc.cu): plan and
// launch a batch on counters the caller supplies, and record an error.
int batch_with_counters(const vr_request* reqs, int n, unsigned* counters, cudaStream_t s)
{
    return batch_impl(reqs, n, counters, s, g_batch_cfg.load());
}

int record_error(int code, const char* msg) { return fail(code, "%s", msg); }

size_t brick_bytes(const VolumeGeom& g, int dtype)
{
    return (size_t)g.nbx * g.nby * g.nbz * kBrickVoxels * elem_size(dtype);
}

size_t table_offset(const VolumeGeom& g, int dtype)
{
    return align_up(brick_bytes(g, dtype), 256);
}

}  // namespace vr

extern "C" {

static_assert(sizeof(vr_request) == 136, "vr_request is 136 bytes in ABI version 2");

int vr_debug_status(unsigned* flags, int clear)
{
#ifdef VR_DEBUG
    if (!flags) return fail(VR_ERR_ARG, "flags is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronising for the check words");
    const bool c = clear != 0;
    *flags = vr::debug_flags_tex_f32(c) | vr::debug_flags_tex_f16(c) | vr::debug_flags_tex_i8(c) |
             vr::debug_flags_tex_f16pair(c) | vr::debug_flags_tex_i8pair(c) |
             vr::debug_flags_batch(c) | vr::debug_flags_integrate(c) |
             vr::debug_flags_object(c);
    return VR_OK;
#else
    (void)clear;
    if (flags) *flags = 0;
    return fail(VR_ERR_UNSUPPORTED, "not a checked build (compile with VR_DEBUG)");
#endif
}

int vr_version(void) { return 2; }

const char* vr_last_error(void) { return g_err.c_str(); }

int vr_volume_bytes(const int64_t dims[3], int dtype, size_t* bytes_out)
{
    vr::VolumeGeom g;
    int rc = check_dims(dims, dtype, &g);
    if (rc) return rc;
    if (!bytes_out) return fail(VR_ERR_ARG, "bytes_out is NULL");
    size_t b = vr::brick_bytes(g, dtype);
    if (dtype == VR_I8) b = vr::table_offset(g, dtype) + 2 * align_up((size_t)g.nz * 4, 256);
    *bytes_out = b;
    return VR_OK;
}

int vr_texture_bytes(const int64_t dims[3], int dtype, int pair, size_t* bytes_out)
{
    vr::VolumeGeom g;
    int rc = check_dims(dims, dtype, &g);
    if (rc) return rc;
    if (!bytes_out) return fail(VR_ERR_ARG, "bytes_out is NULL");
    if (pair && dtype == VR_F32)
        return fail(VR_ERR_UNSUPPORTED, "pair textures hold FP16 or int8 storage only");
    TexLayout L;
    rc = texture_layout(g, pair != 0, &L);
    if (rc) return rc;
    const int format = pair ? (dtype == VR_F16 ? vr::kF16Pair : vr::kI8Pair) : dtype;
    *bytes_out = texture_bytes(g, format, L);
    return VR_OK;
}

int vr_mip_bounds_bytes(const int64_t dims[3], size_t* bytes_out)
{
    vr::VolumeGeom g;
    int rc = check_dims(dims, VR_F32, &g);
    if (rc) return rc;
    if (!bytes_out) return fail(VR_ERR_ARG, "bytes_out is NULL");
    TexLayout L;
    rc = texture_layout(g, false, &L);
    if (rc) return rc;
    *bytes_out = bounds_bytes(g, bound_layout(g, L.shift, L.pitch));
    return VR_OK;
}

int vr_volume_device_bytes(vr_volume vol, size_t* library_bytes, size_t* caller_bytes)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    const vr::Volume* v = reinterpret_cast<const vr::Volume*>(vol);
    size_t lib = 0, caller = 0;
    if (v->has_tex) {
        const bool pair = v->tex_format == vr::kF16Pair || v->tex_format == vr::kI8Pair;
        const int slices = pair ? v->g.nz + 1 : v->g.nz + 2;
        const TexLayout L{slices, v->stack_shift, v->stack_pitch,
                          (slices + (1 << v->stack_shift) - 1) >> v->stack_shift};
        lib += texture_bytes(v->g, v->tex_format, L);
        if (v->bound_array)
            lib += bounds_bytes(v->g, bound_layout(v->g, v->stack_shift, v->stack_pitch));
    }
    if (v->bricks) caller += v->bytes;
    if (v->mask) caller += mask_macrocells(v->g) * sizeof(unsigned long long);
    if (library_bytes) *library_bytes = lib;
    if (caller_bytes) *caller_bytes = caller;
    return VR_OK;
}

int vr_volume_create(const int64_t dims[3], int dtype, const float* src, int src_on_device,
                     void* brick_buf, size_t brick_bytes, void* stream, vr_volume* out)
{
    const NvtxRange nvtx_range("vr_volume_create");
    if (!out) return fail(VR_ERR_ARG, "out is NULL");
    *out = nullptr;
    vr::VolumeGeom g;
    int rc = check_dims(dims, dtype, &g);
    if (rc) return rc;
    size_t need = 0;
    vr_volume_bytes(dims, dtype, &need);
    if (!brick_buf) return fail(VR_ERR_ARG, "brick_buf is NULL");
    if (reinterpret_cast<uintptr_t>(brick_buf) % 256 != 0)
        return fail(VR_ERR_ARG, "brick_buf must be 256-byte aligned");
    if (brick_bytes < need)
        return fail(VR_ERR_OOM, "brick_buf has %zu bytes, %zu needed", brick_bytes, need);
    if (!is_device_ptr(brick_buf)) return fail(VR_ERR_ARG, "brick_buf is not device memory");
    vr::Volume* v = new (std::nothrow) vr::Volume;
    if (!v) return fail(VR_ERR_OOM, "out of host memory");
    std::memset(v, 0, sizeof *v);
    v->g = g;
    v->dtype = dtype;
    v->bricks = brick_buf;
    v->bytes = brick_bytes;
    if (dtype == VR_I8) {
        char* base = static_cast<char*>(brick_buf) + vr::table_offset(g, dtype);
        v->scale = reinterpret_cast<float*>(base);
        v->offset = reinterpret_cast<float*>(base + align_up((size_t)g.nz * 4, 256));
    }
    default_transfer(v);
    if (src) {
        rc = vr_volume_upload(reinterpret_cast<vr_volume>(v), 0, g.nz, src, src_on_device, stream);
        if (rc) {
            delete v;
            return rc;
        }
    }
    *out = reinterpret_cast<vr_volume>(v);
    return VR_OK;
}

int vr_volume_upload(vr_volume vol, int64_t z0, int64_t nplanes, const float* src,
                     int src_on_device, void* stream)
{
    const NvtxRange nvtx_range("vr_volume_upload");
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    if (!src) return fail(VR_ERR_ARG, "src is NULL");
    if (z0 < 0 || nplanes < 1 || z0 + nplanes > v->g.nz)
        return fail(VR_ERR_ARG, "planes [%lld, %lld) outside [0, %d)", (long long)z0,
                    (long long)(z0 + nplanes), v->g.nz);
    if (v->texture_only)
        return fail(VR_ERR_UNSUPPORTED, "the volume's bricks were dropped: it is read-only");
    const float* dsrc = src;
    if (src_on_device) {
        if (!is_device_ptr(src)) return fail(VR_ERR_ARG, "src is not device memory");
    } else {
        dsrc = static_cast<const float*>(host_to_device_ptr(src));
        if (!dsrc) return fail(VR_ERR_ARG, "host src must be page-locked (pinned) memory");
    }
    cudaError_t e = vr::launch_pack(*v, z0, nplanes, dsrc, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "pack launch");
    v->mask_clip = NAN;               // masks are rebuilt by the next composite render
    if (v->has_tex && v->tex_format == VR_F32 && v->stack_shift == 0)
        return copy_texture_planes(v, z0, nplanes, dsrc, static_cast<cudaStream_t>(stream));
    if (v->has_tex)
        return refresh_texture(v, z0, z0 + nplanes, static_cast<cudaStream_t>(stream));
    return VR_OK;
}

int vr_set_transfer(vr_volume vol, const float* rgba_lut, int n, float v_lo, float v_hi,
                    float clip, float term_alpha)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    if (!rgba_lut) return fail(VR_ERR_ARG, "rgba_lut is NULL");
    if (n < 2 || n > VR_MAX_LUT) return fail(VR_ERR_ARG, "table size %d outside [2, %d]", n, VR_MAX_LUT);
    if (!std::isfinite(v_lo) || !std::isfinite(v_hi) || !(v_lo < v_hi))
        return fail(VR_ERR_ARG, "need finite v_lo < v_hi");
    if (std::isnan(clip) || std::isnan(term_alpha)) return fail(VR_ERR_ARG, "clip/term_alpha NaN");
    for (int i = 0; i < n; ++i) {
        for (int c = 0; c < 4; ++c)
            if (!std::isfinite(rgba_lut[4 * i + c]))
                return fail(VR_ERR_ARG, "table entry %d is not finite", i);
        if (rgba_lut[4 * i + 3] < 0.0f || rgba_lut[4 * i + 3] > 1.0f)
            return fail(VR_ERR_ARG, "table alpha %d outside [0, 1]", i);
    }
    std::memcpy(v->lut_raw, rgba_lut, sizeof(float) * 4 * n);
    v->n_lut = n;
    v->v_lo = v_lo;
    v->v_hi = v_hi;
    v->clip = clip;
    v->term_alpha = term_alpha;
    v->lut_valid = false;
    return VR_OK;
}

int vr_render(vr_volume vol, const vr_camera* cams, int n_views, int w, int h, int mode,
              float step, float* out, void* stream)
{
    const NvtxRange nvtx_range("vr_render");
    return render_impl(vol, cams, n_views, w, h, mode, step, out, nullptr, stream);
}

int vr_render_counted(vr_volume vol, const vr_camera* cams, int n_views, int w, int h, int mode,
                      float step, float* out, unsigned long long* d_samples, void* stream)
{
    const NvtxRange nvtx_range("vr_render_counted");
    if (!d_samples) return fail(VR_ERR_ARG, "d_samples is NULL");
    return render_impl(vol, cams, n_views, w, h, mode, step, out, d_samples, stream);
}

int vr_render_object_order(vr_volume vol, const vr_camera* cams, int n_views, int w, int h,
                           int mode, float step, float* out, unsigned long long* d_samples,
                           void* stream)
{
    const NvtxRange nvtx_range("vr_render_object_order");
    if (mode == VR_COMPOSITE || mode == VR_SUM)
        return fail(VR_ERR_ARG, "object-order rendering takes MIP only (mode %d)", mode);
    vr::MarchParams p;
    vr::TexParams tp;
    int rc = prepare(vol, cams, n_views, w, h, mode, step, out, d_samples, &p, &tp);
    if (rc) return rc;
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    if (v->texture_only)
        return fail(VR_ERR_UNSUPPORTED, "object-order rendering reads the bricks, which were dropped");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = vr::launch_render_init(out, (size_t)n_views * w * h, VR_MIP, s);
    if (e != cudaSuccess) return cuda_fail(e, "init launch");
    const size_t per_view = (size_t)w * h;
    for (int v0 = 0; v0 < n_views; v0 += vr::kMaxViewsPerLaunch) {
        const int nv = std::min(vr::kMaxViewsPerLaunch, n_views - v0);
        p.n_views = nv;
        std::memcpy(p.cams, cams + v0, sizeof(vr_camera) * nv);
        p.out = out + per_view * v0;
        e = vr::launch_object(p, tp.k_max, v->dtype, s);
        if (e != cudaSuccess) return cuda_fail(e, "object-order launch");
    }
    return VR_OK;
}

int vr_volume_attach_texture(vr_volume vol, void* stream)
{
    const NvtxRange nvtx_range("vr_volume_attach_texture");
    return attach_texture(vol, false, stream);
}

int vr_volume_attach_pair_texture(vr_volume vol, void* stream)
{
    const NvtxRange nvtx_range("vr_volume_attach_pair_texture");
    return attach_texture(vol, true, stream);
}

int vr_volume_attach_mip_bounds(vr_volume vol, void* stream)
{
    const NvtxRange nvtx_range("vr_volume_attach_mip_bounds");
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    return attach_bounds(reinterpret_cast<vr::Volume*>(vol), static_cast<cudaStream_t>(stream));
}

int vr_volume_detach_mip_bounds(vr_volume vol)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    release_bounds(reinterpret_cast<vr::Volume*>(vol));
    return VR_OK;
}

int vr_volume_detach_texture(vr_volume vol)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    if (v->texture_only)
        return fail(VR_ERR_UNSUPPORTED, "the texture is the volume's only copy (bricks dropped)");
    release_texture(v);
    return VR_OK;
}

int vr_volume_drop_bricks(vr_volume vol)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    if (v->texture_only) return VR_OK;
    if (!v->has_tex) return fail(VR_ERR_UNSUPPORTED, "the volume has no texture storage");
    v->texture_only = true;
    v->bricks = nullptr;
    if (std::isnan(v->mask_clip)) v->mask = nullptr;   // never built: nothing to keep
    return VR_OK;
}

int vr_render_init(float* out, int n_views, int w, int h, int mode, void* stream)
{
    if (!out) return fail(VR_ERR_ARG, "out is NULL");
    if (n_views < 1 || w < 1 || h < 1) return fail(VR_ERR_ARG, "empty image set");
    if (mode != VR_MIP && mode != VR_COMPOSITE && mode != VR_SUM)
        return fail(VR_ERR_ARG, "unknown mode %d", mode);
    if (reinterpret_cast<uintptr_t>(out) % out_alignment(mode) != 0)
        return fail(VR_ERR_ARG, "out must be %d-byte aligned", out_alignment(mode));
    if (!is_device_ptr(out)) return fail(VR_ERR_ARG, "out is not device memory of this device");
    cudaError_t e = vr::launch_render_init(out, (size_t)n_views * w * h, mode,
                                           static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? VR_OK : cuda_fail(e, "init launch");
}

int vr_integrate_partials(const float* partials, int n_parts, const vr_camera* cams,
                          int n_views, int w, int h, int mode, float* out, void* stream)
{
    const NvtxRange nvtx_range("vr_integrate_partials");
    if (!partials || !out) return fail(VR_ERR_ARG, "partials or out is NULL");
    if (!cams) return fail(VR_ERR_ARG, "cams is NULL");
    if (n_parts < 1) return fail(VR_ERR_ARG, "n_parts = %d < 1", n_parts);
    if (n_views < 1 || w < 1 || h < 1 || w > 65536 || h > 65536)
        return fail(VR_ERR_ARG, "image set %d x %d x %d is empty or too large", n_views, w, h);
    if (mode != VR_MIP && mode != VR_COMPOSITE && mode != VR_SUM)
        return fail(VR_ERR_ARG, "unknown mode %d", mode);
    if (reinterpret_cast<uintptr_t>(partials) % out_alignment(mode) != 0 ||
        reinterpret_cast<uintptr_t>(out) % out_alignment(mode) != 0)
        return fail(VR_ERR_ARG, "partials and out must be %d-byte aligned", out_alignment(mode));
    if (!is_device_ptr(partials) || !is_device_ptr(out))
        return fail(VR_ERR_ARG, "partials and out must be device memory of this device");
    const size_t pixels = (size_t)n_views * w * h;
    const size_t ch = mode == VR_COMPOSITE ? 4 : 1;
    const float* p_end = partials + pixels * ch * (size_t)n_parts;
    if (out < p_end && partials < out + pixels * ch)
        return fail(VR_ERR_ARG, "out overlaps the partial images");
    for (int i = 0; i < n_views; ++i) {
        const vr_camera& c = cams[i];
        if (c.proj != VR_ORTHO && c.proj != VR_PERSP)
            return fail(VR_ERR_ARG, "camera %d: unknown projection %d", i, c.proj);
        if (!finite3(c.eye) || !finite3(c.fwd) || !finite3(c.du) || !finite3(c.dv))
            return fail(VR_ERR_ARG, "camera %d: non-finite parameters", i);
    }
    vr::IntegrateParams p;
    std::memset(&p, 0, sizeof p);
    p.n_parts = n_parts;
    p.w = w;
    p.h = h;
    p.part_stride = pixels;
    const size_t per_view = (size_t)w * h * ch;
    for (int v0 = 0; v0 < n_views; v0 += vr::kMaxViewsPerLaunch) {
        const int nv = std::min(vr::kMaxViewsPerLaunch, n_views - v0);
        p.n_views = nv;
        std::memcpy(p.cams, cams + v0, sizeof(vr_camera) * nv);
        p.partials = partials + per_view * v0;
        p.out = out + per_view * v0;
        cudaError_t e = vr::launch_integrate(p, mode, static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail(e, "integration launch");
    }
    return VR_OK;
}

int vr_render_part(vr_volume part, const int64_t full_dims[3], int64_t z_first,
                   int64_t cell_lo, int64_t cell_hi, const vr_camera* cams, int n_views,
                   int w, int h, int mode, float step, int sweep, float* out,
                   unsigned long long* d_samples, void* stream)
{
    const NvtxRange nvtx_range("vr_render_part");
    if (!part) return fail(VR_ERR_ARG, "volume is NULL");
    vr::Volume* v = reinterpret_cast<vr::Volume*>(part);
    if (!full_dims) return fail(VR_ERR_ARG, "full_dims is NULL");
    if (!v->has_tex) return fail(VR_ERR_UNSUPPORTED, "part rendering needs texture storage");
    if (full_dims[0] != v->g.nx || full_dims[1] != v->g.ny)
        return fail(VR_ERR_ARG, "the part's nx, ny differ from the cube's");
    if (z_first < 0 || z_first + v->g.nz > full_dims[2] || full_dims[2] > (1 << 20))
        return fail(VR_ERR_ARG, "part planes [%lld, %lld) outside the cube's %lld",
                    (long long)z_first, (long long)(z_first + v->g.nz), (long long)full_dims[2]);
    if (cell_lo < z_first || cell_hi > z_first + v->g.nz - 1 || cell_lo > cell_hi)
        return fail(VR_ERR_ARG, "cells [%lld, %lld) are not within the part's planes [%lld, %lld]",
                    (long long)cell_lo, (long long)cell_hi, (long long)z_first,
                    (long long)(z_first + v->g.nz - 1));
    if (sweep != 1 && sweep != -1 && sweep != 0)
        return fail(VR_ERR_ARG, "sweep must be +1, -1 or 0");
    vr::MarchParams p;
    vr::TexParams tp;
    int rc = prepare(part, cams, n_views, w, h, mode, step, out, d_samples, &p, &tp);
    if (rc) return rc;
    // the whole cube's box and sample bound; the part's cells and slices
    const double hz = full_dims[2] - 1.0;
    const double hx = v->g.nx - 1.0, hy = v->g.ny - 1.0;
    const double diag = std::sqrt(hx * hx + hy * hy + hz * hz);
    if (diag / step + 2.0 >= 16777216.0)
        return fail(VR_ERR_ARG, "step %g too small: a ray could take 2^24 samples", (double)step);
    p.hiz = (float)hz;
    tp.k_max = (int)(diag / step) + 2;
    p.part_lo = cell_lo == 0 ? INT_MIN : (int)cell_lo;
    p.part_hi = cell_hi == full_dims[2] - 1 ? INT_MAX : (int)cell_hi;
    p.slice_base = (int)z_first;
    p.sweep = sweep;
    // masks only where they hold for the clip: nothing rebuilds them here
    // (a part's bricks may already hold another part; see
    // vr_volume_build_masks)
    const bool masks_valid = v->mask && !std::isnan(v->mask_clip) && !(v->clip < v->mask_clip);
    if (mode != VR_COMPOSITE || !masks_valid) p.mask = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t per_view = (size_t)w * h * (mode == VR_COMPOSITE ? 4 : 1);
    for (int v0 = 0; v0 < n_views; v0 += vr::kMaxViewsPerLaunch) {
        const int nv = std::min(vr::kMaxViewsPerLaunch, n_views - v0);
        p.n_views = nv;
        std::memcpy(p.cams, cams + v0, sizeof(vr_camera) * nv);
        p.out = out + per_view * v0;
        cudaError_t e = vr::launch_part(p, tp, v->tex_format, mode, s);
        if (e != cudaSuccess) return cuda_fail(e, "part launch");
    }
    return VR_OK;
}

int vr_volume_build_masks(vr_volume vol, void* stream)
{
    const NvtxRange nvtx_range("vr_volume_build_masks");
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    if (!v->mask) return fail(VR_ERR_UNSUPPORTED, "no masks are attached");
    if (v->texture_only)
        return fail(VR_ERR_UNSUPPORTED, "masks are built from the bricks, which were dropped");
    cudaError_t e = vr::launch_masks(*v, v->clip, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "mask launch");
    v->mask_clip = v->clip;
    return VR_OK;
}

int vr_volume_mask_bytes(vr_volume vol, size_t* bytes_out)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    if (!bytes_out) return fail(VR_ERR_ARG, "bytes_out is NULL");
    const vr::Volume* v = reinterpret_cast<const vr::Volume*>(vol);
    *bytes_out = sizeof(unsigned long long) * mask_macrocells(v->g);
    return VR_OK;
}

int vr_volume_attach_masks(vr_volume vol, void* buf, size_t bytes)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    if (!buf) {
        v->mask = nullptr;
        return VR_OK;
    }
    if (v->texture_only)
        return fail(VR_ERR_UNSUPPORTED, "masks are built from the bricks, which were dropped");
    const size_t nm = mask_macrocells(v->g);
    if (nm > 0x7fffffffu || (v->g.ny >> vr::kMacroShift) + 1 > 65535)
        return fail(VR_ERR_UNSUPPORTED, "cube too large for empty-space masks");
    if (reinterpret_cast<uintptr_t>(buf) % 16 != 0)
        return fail(VR_ERR_ARG, "mask buffer must be 16-byte aligned");
    if (bytes < nm * sizeof(unsigned long long))
        return fail(VR_ERR_OOM, "mask buffer has %zu bytes, %zu needed", bytes,
                    nm * sizeof(unsigned long long));
    if (!is_device_ptr(buf)) return fail(VR_ERR_ARG, "mask buffer is not device memory");
    v->mask = static_cast<unsigned long long*>(buf);
    v->mask_clip = NAN;                       // built by the next composite render
    v->mnx = (v->g.nx >> vr::kMacroShift) + 1;
    v->mny = (v->g.ny >> vr::kMacroShift) + 1;
    v->mnz = (v->g.nz >> vr::kMacroShift) + 1;
    return VR_OK;
}

size_t vr_batch_workspace_bytes(void)
{
    return align_up(sizeof(unsigned) * vr::kBatchWords, 256);
}

namespace {

int check_batch_args(const vr_request* reqs, int n, void* workspace, size_t ws_bytes)
{
    if (n < 0) return fail(VR_ERR_ARG, "n = %d < 0", n);
    if (n == 0) return VR_OK;
    if (!reqs) return fail(VR_ERR_ARG, "reqs is NULL");
    if (!workspace) return fail(VR_ERR_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) % 16 != 0)
        return fail(VR_ERR_ARG, "workspace must be 16-byte aligned");
    if (ws_bytes < vr_batch_workspace_bytes())
        return fail(VR_ERR_OOM, "workspace has %zu bytes, %zu needed", ws_bytes,
                    vr_batch_workspace_bytes());
    if (!is_device_ptr(workspace)) return fail(VR_ERR_ARG, "workspace is not device memory");
    return VR_OK;
}

}  // namespace

int vr_render_batch(const vr_request* reqs, int n, void* workspace, size_t ws_bytes,
                    void* stream)
{
    const NvtxRange nvtx_range("vr_render_batch");
    const int rc = check_batch_args(reqs, n, workspace, ws_bytes);
    if (rc || n == 0) return rc;
    return batch_impl(reqs, n, static_cast<unsigned*>(workspace),
                      static_cast<cudaStream_t>(stream), g_batch_cfg.load());
}

int vr_batch_tune_count(void) { return vr::kNumBatchShapes; }

int vr_batch_tune_describe(int cfg, int* tile_x, int* tile_y, int* packet_x, int* packet_y)
{
    if (cfg < 0 || cfg >= vr::kNumBatchShapes)
        return fail(VR_ERR_ARG, "batch configuration %d out of range", cfg);
    const vr::BatchShape& S = vr::kBatchShapes[cfg];
    if (tile_x) *tile_x = S.tx;
    if (tile_y) *tile_y = S.ty;
    if (packet_x) *packet_x = S.px;
    if (packet_y) *packet_y = S.py;
    return VR_OK;
}

int vr_set_batch_config(int cfg)
{
    if (cfg < 0 || cfg >= vr::kNumBatchShapes)
        return fail(VR_ERR_ARG, "batch configuration %d out of range", cfg);
    g_batch_cfg.store(cfg);
    return VR_OK;
}

int vr_get_batch_config(void) { return g_batch_cfg.load(); }

int vr_batch_autotune(const vr_request* reqs, int n, void* workspace, size_t ws_bytes,
                      void* stream, int* best_cfg, float* best_ms)
{
    const NvtxRange nvtx_range("vr_batch_autotune");
    int rc = check_batch_args(reqs, n, workspace, ws_bytes);
    if (rc) return rc;
    if (n == 0) {
        if (best_cfg) *best_cfg = g_batch_cfg.load();
        if (best_ms) *best_ms = -1.0f;
        return VR_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned* ws = static_cast<unsigned*>(workspace);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "event");
    }
    int best = -1;
    float best_t = 0.0f;
    for (int c = 0; c < vr::kNumBatchShapes && rc == VR_OK; ++c) {
        float t = 1e30f;
        for (int it = 0; it < 3 && rc == VR_OK; ++it) {    // first run warms up
            cudaEventRecord(e0, s);
            rc = batch_impl(reqs, n, ws, s, c);
            cudaEventRecord(e1, s);
            const cudaError_t e = cudaEventSynchronize(e1);
            if (rc == VR_OK && e != cudaSuccess) rc = cuda_fail(e, "batch autotune");
            float ms = 0.0f;
            if (rc == VR_OK) cudaEventElapsedTime(&ms, e0, e1);
            if (it > 0 && ms < t) t = ms;
        }
        if (rc == VR_OK && (best < 0 || t < best_t)) {
            best = c;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    g_batch_cfg.store(best);
    if (best_cfg) *best_cfg = best;
    if (best_ms) *best_ms = best_t;
    return VR_OK;
}

int vr_tune_count(void) { return vr::tex_shape_count(); }

int vr_tune_describe(int cfg, int* block_x, int* block_y, int* packet_x, int* packet_y,
                     int* min_blocks)
{
    if (cfg < 0 || cfg >= vr::tex_shape_count())
        return fail(VR_ERR_ARG, "launch configuration %d out of range", cfg);
    int bx, by, px, py, mb;
    vr::tex_shape(cfg, &bx, &by, &px, &py, &mb);
    if (block_x) *block_x = bx;
    if (block_y) *block_y = by;
    if (packet_x) *packet_x = px;
    if (packet_y) *packet_y = py;
    if (min_blocks) *min_blocks = mb;
    return VR_OK;
}

int vr_set_launch_config(vr_volume vol, int mode, int cfg)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    if (mode != VR_MIP && mode != VR_COMPOSITE && mode != VR_SUM)
        return fail(VR_ERR_ARG, "unknown mode %d", mode);
    if (cfg < 0 || cfg >= vr::tex_shape_count())
        return fail(VR_ERR_ARG, "launch configuration %d out of range", cfg);
    reinterpret_cast<vr::Volume*>(vol)->cfg[mode] = cfg;
    return VR_OK;
}

int vr_autotune(vr_volume vol, const vr_camera* cams, int n_views, int w, int h, int mode,
                float step, float* out, void* stream, int* best_cfg, float* best_ms)
{
    const NvtxRange nvtx_range("vr_autotune");
    vr::MarchParams p;
    vr::TexParams tp;
    int rc = prepare(vol, cams, n_views, w, h, mode, step, out, nullptr, &p, &tp);
    if (rc) return rc;
    vr::Volume* v = reinterpret_cast<vr::Volume*>(vol);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!v->has_tex) {   // only the texture kernel has shapes to choose from
        if (best_cfg) *best_cfg = v->cfg[mode];
        if (best_ms) *best_ms = -1.0f;
        return VR_OK;
    }
    rc = ensure_masks(v, mode, s, &p);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "event");
    }
    int best = -1;
    float best_t = 0.0f;
    for (int c = 0; c < vr::tex_shape_count() && rc == VR_OK; ++c) {
        float t = 1e30f;
        for (int it = 0; it < 3 && rc == VR_OK; ++it) {    // first run warms up
            cudaEventRecord(e0, s);
            rc = launch_views(v, p, tp, mode, c, cams, n_views, out, s);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "autotune");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (it > 0 && ms < t) t = ms;
        }
        if (rc == VR_OK && (best < 0 || t < best_t)) {
            best = c;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    v->cfg[mode] = best;
    if (best_cfg) *best_cfg = best;
    if (best_ms) *best_ms = best_t;
    return VR_OK;
}

int vr_volume_destroy(vr_volume vol)
{
    if (vol) release_texture(reinterpret_cast<vr::Volume*>(vol));
    delete reinterpret_cast<vr::Volume*>(vol);
    return VR_OK;
}

int vr_volume_info(vr_volume vol, int64_t dims[3], int* dtype, void** brick_buf)
{
    if (!vol) return fail(VR_ERR_ARG, "volume is NULL");
    const vr::Volume* v = reinterpret_cast<const vr::Volume*>(vol);
    if (dims) {
        dims[0] = v->g.nx;
        dims[1] = v->g.ny;
        dims[2] = v->g.nz;
    }
    if (dtype) *dtype = v->dtype;
    if (brick_buf) *brick_buf = v->bricks;
    return VR_OK;
}

}  // extern "C"
