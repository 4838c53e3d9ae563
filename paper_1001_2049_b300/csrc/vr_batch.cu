// vr_batch.cu -- many render requests (mixed cubes, storage types,
// resolutions, modes and transfer functions) in one persistent launch.
//
// The paper's scheduling module maps the available tasks onto the computing
// resources (Fig. 1 caption, §3.1 module 1); on one GPU the tasks are the
// ray tiles (256 rays, in one of kBatchShapes) of every requested view and
// the resources are the SMs.
// The launch puts about as many blocks as fit on the device at once; each
// block repeatedly takes the next tile from a work counter in the caller's
// workspace (an atomic add, no waiting on anything), renders it with the
// same per-ray march as the single-view kernels (vr_ray.cuh), and counts the
// tile as done in its request's counter.  The block that completes a
// request's last tile optionally writes the request's `done` word (device or
// mapped host memory) after a system-scope fence, so a caller can see
// requests finish while the rest of the batch is still running.
#include "vr_internal.h"
#include "vr_ray.cuh"

namespace vr {
namespace {

constexpr int kThreads = 256;             // one ray per thread, a tile per block
#ifndef VR_BATCH_MIN_BLOCKS
#define VR_BATCH_MIN_BLOCKS 4     // resident blocks per SM the registers must allow
#endif
// Pair texels hold half the corner registers: six blocks (48 warps) per SM,
// measured faster than four for both modes (a 1024^3 FP16 pair cube, 32 views
// of 1024^2: 65 -> 56 ms).
#ifndef VR_BATCH_PAIR_MIN_BLOCKS
#define VR_BATCH_PAIR_MIN_BLOCKS 6
#endif

// Find the request whose items contain `item` (first_item ascending).
__device__ __forceinline__ int find_request(const BatchParams& B, int item)
{
    int lo = 0, hi = B.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.req[mid].first_item <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Requests on volumes with texture storage run the single-view kernels'
// march specialised per texel format, mode and plane stacking (one switch,
// uniform over a block).  Requests on volumes without texture storage gather
// from the bricks with the mode and storage type as run-time values.

struct AccRT {
    float r = 0.0f, g = 0.0f, b = 0.0f, A = 0.0f, m;
    int mode;
    __device__ explicit AccRT(int md) : m(md == VR_MIP ? -INFINITY : 0.0f), mode(md) {}

    __device__ __forceinline__ bool add(const BatchReq& P, const float4* __restrict__ lut, float s)
    {
        if (mode == VR_MIP) {
            m = fmaxf(m, s);
            return false;
        }
        if (mode == VR_SUM) {
            m = fmaf(s, P.step, m);
            return false;
        }
        if (!(s >= P.clip)) return false;
        const float x = fminf(fmaxf((s - P.v_lo) * P.lut_scale, 0.0f), P.lut_max);
        const int i = min((int)x, P.n_lut - 2);
        const float f = x - (float)i;
        const float4 a = lut[i], c = lut[i + 1];
        const float alpha = ray::lerpf(a.w, c.w, f);
        const float wgt = (1.0f - A) * alpha;
        r = fmaf(wgt, ray::lerpf(a.x, c.x, f), r);
        g = fmaf(wgt, ray::lerpf(a.y, c.y, f), g);
        b = fmaf(wgt, ray::lerpf(a.z, c.z, f), b);
        A += wgt;
        return A >= P.term_alpha;
    }
};

// Brick path: eight loads per sample (storage type at run time).
__device__ __forceinline__ int march_bricks_rt(const BatchReq& P, const float4* __restrict__ lut,
                                               const ray::Ray& r, AccRT& acc)
{
    int k = 0;
    float kf = 0.0f;
    for (; k < r.K; ++k, kf += 1.0f) {
        const float t = fmaf(kf, P.step, r.te);
        const float qx = fminf(fmaxf(fmaf(t, r.dx, r.ox), 0.0f), P.hix);
        const float qy = fminf(fmaxf(fmaf(t, r.dy, r.oy), 0.0f), P.hiy);
        const float qz = fminf(fmaxf(fmaf(t, r.dz, r.oz), 0.0f), P.hiz);
        float s;
        if (P.dtype == VR_F32)
            s = ray::sample_bricks<VR_F32>(P, qx, qy, qz);
        else if (P.dtype == VR_F16)
            s = ray::sample_bricks<VR_F16>(P, qx, qy, qz);
        else
            s = ray::sample_bricks<VR_I8>(P, qx, qy, qz);
        if (acc.add(P, lut, s)) {
            ++k;
            break;
        }
    }
    return k;
}

// Texture path, specialised: the march of the single-view texture kernel for
// one texel format, mode and plane stacking (template parameters), so a
// block renders its tile with exactly the code the per-view kernel runs.
template <int DT, int MODE, bool STACK>
__device__ __forceinline__ unsigned tex_pixel(const BatchReq& q, const BatchTex& T,
                                              const float4* __restrict__ lut, int px, int py)
{
    const ray::Ray r = ray::setup_ray(q, q.cam, px, py, q.k_max);
    ray::Acc<MODE> acc;
    const int k = ray::march_tex<DT, MODE, STACK, true>(q, T, lut, r, acc);
    const size_t pix = (size_t)(py - q.row0) * q.w + px;
    if (!ray::debug_ok(py >= q.row0 && pix < (size_t)(q.row_end - q.row0) * q.w, 1)) {
    } else if (MODE == VR_COMPOSITE)
        reinterpret_cast<float4*>(q.out)[pix] = make_float4(acc.r, acc.g, acc.b, acc.A);
    else
        q.out[pix] = acc.m;
    return (unsigned)k;
}

// Kind of a textured request: (texel format, mode, stacked planes).
__host__ __device__ constexpr int tex_kind(int format, int mode, bool stack)
{
    return (format * 3 + mode) * 2 + (stack ? 1 : 0);
}

// One switch over the kinds of a launch class (uniform over the block: a
// tile belongs to one request); each case is the specialised march of one
// kind.  PAIR: the pair texel formats, else the plain ones.
template <bool PAIR>
__device__ __forceinline__ unsigned tex_pixel_any(const BatchReq& q, const BatchTex& T,
                                                  const float4* __restrict__ lut, int px, int py)
{
#define VR_KIND(F, M)                                                              \
    case tex_kind(F, M, false): return tex_pixel<F, M, false>(q, T, lut, px, py);  \
    case tex_kind(F, M, true): return tex_pixel<F, M, true>(q, T, lut, px, py);
#define VR_FORMAT(F) VR_KIND(F, VR_MIP) VR_KIND(F, VR_COMPOSITE) VR_KIND(F, VR_SUM)
    if constexpr (PAIR) {
        switch (tex_kind(T.format, q.mode, T.stack_shift > 0)) {
            VR_FORMAT(kF16Pair)
            VR_FORMAT(kI8Pair)
        default: return 0;
        }
    } else {
        switch (tex_kind(T.format, q.mode, T.stack_shift > 0)) {
            VR_FORMAT(VR_F32)
            VR_FORMAT(VR_F16)
            VR_FORMAT(VR_I8)
        default: return 0;
        }
    }
#undef VR_FORMAT
#undef VR_KIND
}

// CLS (BatchClass): every request of the launch is of one class, so each
// kernel instance compiles one fetch path: bricks (run-time storage type) or
// texture (specialised per kind), plain and pair texel formats apart.  CFG: the tile and ray-packet shape
// (kBatchShapes), chosen by vr_batch_autotune.
template <int CLS, int CFG>
__global__ void __launch_bounds__(kThreads, CLS == kBatchTexPair ? VR_BATCH_PAIR_MIN_BLOCKS
                                                                 : VR_BATCH_MIN_BLOCKS)
    batch_kernel(const __grid_constant__ BatchParams B,
                                                         unsigned* __restrict__ ws)
{
    constexpr BatchShape S = kBatchShapes[CFG];
    constexpr int wpr = S.tx / S.px;               // warps per row of packets
    static_assert(S.tx * S.ty == kThreads && S.px * S.py == 32 && S.tx % S.px == 0 &&
                      S.ty % S.py == 0,
                  "a tile is 256 rays in warp packets");
    __shared__ float4 s_lut[VR_MAX_LUT];
    __shared__ int s_item;
    __shared__ int s_lut_slot;
    unsigned* next_item = ws;           // work counter
    unsigned* tiles_done = ws + 1;      // one per request
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_lut_slot = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(next_item, 1u);
        __syncthreads();
        const int item = s_item;
        const int lut_slot_loaded = s_lut_slot;
        __syncthreads();                 // s_item / s_lut_slot are rewritten below
        if (item >= B.total_items) break;
        const int ri = find_request(B, item);
        const BatchReq& q = B.req[ri];
        if (q.mode == VR_COMPOSITE && q.lut_slot != lut_slot_loaded) {
            for (int i = threadIdx.x; i < q.n_lut; i += kThreads)
                s_lut[i] = B.lut[q.lut_slot][i];
            if (threadIdx.x == 0) s_lut_slot = q.lut_slot;
            __syncthreads();
        }
        const int t = item - q.first_item;
        if (!ray::debug_ok(t >= 0 && t < q.n_tiles, 8)) continue;
        const int tx = t % q.tiles_x, ty = t / q.tiles_x;
        const int px = tx * S.tx + (warp % wpr) * S.px + (lane % S.px);
        const int py = q.row0 + ty * S.ty + (warp / wpr) * S.py + (lane / S.px);
        unsigned count = 0;
        if (px < q.w && py < q.row_end) {
            if constexpr (CLS == kBatchTex || CLS == kBatchTexPair) {
                count = tex_pixel_any<CLS == kBatchTexPair>(q, B.tex[q.tex_slot], s_lut, px, py);
            } else {
                const ray::Ray r = ray::setup_ray(q, q.cam, px, py, q.k_max);
                AccRT acc(q.mode);
                count = (unsigned)march_bricks_rt(q, s_lut, r, acc);
                const size_t pix = (size_t)(py - q.row0) * q.w + px;
                if (!ray::debug_ok(pix < (size_t)(q.row_end - q.row0) * q.w, 1)) {
                } else if (q.mode == VR_COMPOSITE)
                    reinterpret_cast<float4*>(q.out)[pix] =
                        make_float4(acc.r, acc.g, acc.b, acc.A);
                else
                    q.out[pix] = acc.m;
            }
        }
        if (q.samples) {
            const unsigned tot = __reduce_add_sync(0xffffffffu, count);
            if (lane == 0 && tot) atomicAdd(q.samples, (unsigned long long)tot);
        }
        // every thread's pixel of this tile is written: count the tile
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned done = atomicAdd(&tiles_done[ri], 1u) + 1u;
            if (done == (unsigned)q.n_tiles && q.done) {
                __threadfence_system();
                *reinterpret_cast<volatile unsigned*>(q.done) = q.done_value;
            }
        }
    }
}

}  // namespace

namespace {

// The kernel instance of a (class, shape) pair.
template <int CFG>
const void* kernel_of_shape(int cls)
{
    return cls == kBatchTex       ? reinterpret_cast<const void*>(batch_kernel<kBatchTex, CFG>)
           : cls == kBatchTexPair ? reinterpret_cast<const void*>(batch_kernel<kBatchTexPair, CFG>)
                                  : reinterpret_cast<const void*>(batch_kernel<kBatchBricks, CFG>);
}

const void* batch_kernel_of(int cls, int cfg)
{
    switch (cfg) {
    case 1: return kernel_of_shape<1>(cls);
    case 2: return kernel_of_shape<2>(cls);
    case 3: return kernel_of_shape<3>(cls);
    case 4: return kernel_of_shape<4>(cls);
    case 5: return kernel_of_shape<5>(cls);
    default: return kernel_of_shape<0>(cls);
    }
}
static_assert(kNumBatchShapes == 6, "batch_kernel_of lists every shape");

}  // namespace

cudaError_t launch_batch(const BatchParams& b, unsigned* ws, int grid, int cls, int cfg,
                         cudaStream_t s)
{
    // the counters start at zero for every launch (stream-ordered, capturable)
    cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(unsigned) * (1 + b.n), s);
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<BatchParams*>(&b), &ws};
    return cudaLaunchKernel(batch_kernel_of(cls, cfg), dim3((unsigned)grid), dim3(kThreads),
                            args, 0, s);
}

int batch_blocks_per_sm(int cls, int cfg)
{
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel_of(cls, cfg),
                                                                  kThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

// the checked build's device word of this translation unit
VR_DEBUG_ACCESSOR(debug_flags_batch)

}  // namespace vr
