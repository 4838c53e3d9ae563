// vr_batch.cu -- many render requests (mixed cubes, storage types,
// resolutions, modes and transfer functions) in one persistent launch.
//
// The paper's scheduling module maps the available tasks onto the computing
// resources (Fig. 1 caption, §3.1 module 1); on one GPU the tasks are the
// 16 x 16 ray tiles of every requested view and the resources are the SMs.
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

constexpr int kTile = 16;
constexpr int kThreads = kTile * kTile;
#ifndef VR_BATCH_MIN_BLOCKS
#define VR_BATCH_MIN_BLOCKS 4     // resident blocks per SM the registers must allow
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

// The batched kernel serves any mix of storage types and modes in one
// launch, so its march takes the mode, the storage type and the number of
// texture groups as run-time values (uniform over a block: the branches on
// them do not diverge) instead of template parameters; only the two fetch
// paths, textures and bricks, are separate code.

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

// One plane's 2 x 2 corners: float texels (f32, f16) or int8 codes decoded
// with the plane's scale and offset.
__device__ __forceinline__ float4 plane_rt(const BatchTex& T, int z, float x, float y, bool i8)
{
    const int g = T.n_groups > 1 ? min(z / (kMaxLayers - 1), T.n_groups - 1) : 0;
    const cudaTextureObject_t t = T.tex[g];
    const int l = z - g * (kMaxLayers - 1);
    if (!i8) return ray::gather<VR_F32>(t, l, x, y);
    const float4 q = ray::gather<VR_I8>(t, l, x, y);
    const float sc = __ldg(T.scale + z), of = __ldg(T.offset + z);
    return make_float4(fmaf(q.x, sc, of), fmaf(q.y, sc, of), fmaf(q.z, sc, of),
                       fmaf(q.w, sc, of));
}

// Both planes of a cell: one gather for the pair formats, two otherwise.
__device__ __forceinline__ void cell_rt(const BatchTex& T, int z, float x, float y, float4& c0,
                                        float4& c1)
{
    if (T.format >= kF16Pair) {
        const int sub = z & ((1 << T.stack_shift) - 1);
        const uint4 p = ray::gather_u32(T.tex[0], z >> T.stack_shift, x,
                                        y + (float)(sub * T.stack_pitch + 1));
        if (T.format == kF16Pair) {
            c0 = make_float4(ray::half_bits(p.x), ray::half_bits(p.y), ray::half_bits(p.z),
                             ray::half_bits(p.w));
            c1 = make_float4(ray::half_bits(p.x >> 16), ray::half_bits(p.y >> 16),
                             ray::half_bits(p.z >> 16), ray::half_bits(p.w >> 16));
        } else {
            const float s0 = __ldg(T.scale + z), o0 = __ldg(T.offset + z);
            const float s1 = __ldg(T.scale + z + 1), o1 = __ldg(T.offset + z + 1);
            c0 = make_float4(fmaf(ray::code_lo(p.x), s0, o0), fmaf(ray::code_lo(p.y), s0, o0),
                             fmaf(ray::code_lo(p.z), s0, o0), fmaf(ray::code_lo(p.w), s0, o0));
            c1 = make_float4(fmaf(ray::code_hi(p.x), s1, o1), fmaf(ray::code_hi(p.y), s1, o1),
                             fmaf(ray::code_hi(p.z), s1, o1), fmaf(ray::code_hi(p.w), s1, o1));
        }
    } else {
        const bool i8 = T.format == VR_I8;
        c0 = plane_rt(T, z, x, y, i8);
        c1 = plane_rt(T, z + 1, x, y, i8);
    }
}

__device__ __forceinline__ void next_rt(const BatchTex& T, const ray::Geo& c, const float4& c0,
                                        const float4& c1, const ray::Geo& n, float4& n0,
                                        float4& n1)
{
    if (n.gx == c.gx && n.gy == c.gy) {
        if (n.iz == c.iz) {
            n0 = c0;
            n1 = c1;
            return;
        }
        if (T.format < kF16Pair && n.iz == c.iz + 1) {
            n0 = c1;
            n1 = plane_rt(T, n.iz + 1, n.gx, n.gy, T.format == VR_I8);
            return;
        }
    }
    cell_rt(T, n.iz, n.gx, n.gy, n0, n1);
}

// Texture path: as ray::march_tex (pipelined one sample ahead, corners reused).
__device__ __forceinline__ int march_tex_rt(const BatchReq& P, const BatchTex& T,
                                            const float4* __restrict__ lut, const ray::Ray& r,
                                            AccRT& acc)
{
    if (r.K <= 0) return 0;
    int k = 0;
    ray::Geo ga = ray::geo(P, r, 0.0f), gb;
    float4 a0, a1, b0, b1;
    cell_rt(T, ga.iz, ga.gx, ga.gy, a0, a1);
    float kf = 1.0f;
    for (;;) {
        gb = ray::geo(P, r, kf);
        next_rt(T, ga, a0, a1, gb, b0, b1);
        ++k;
        if (acc.add(P, lut, ray::interp(a0, a1, ga)) || k >= r.K) break;
        kf += 1.0f;
        ga = ray::geo(P, r, kf);
        next_rt(T, gb, b0, b1, ga, a0, a1);
        ++k;
        if (acc.add(P, lut, ray::interp(b0, b1, gb)) || k >= r.K) break;
        kf += 1.0f;
    }
    return k;
}

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
// one texel format, mode and group count (template parameters), so a block
// renders its tile with exactly the code the per-view kernel runs.
template <int DT, int MODE, bool MULTI>
__device__ __forceinline__ unsigned tex_pixel(const BatchReq& q, const BatchTex& T,
                                              const float4* __restrict__ lut, int px, int py)
{
    const ray::Ray r = ray::setup_ray(q, q.cam, px, py, q.k_max);
    ray::Acc<MODE> acc;
    const int k = ray::march_tex<DT, MODE, MULTI>(q, T, lut, r, acc);
    const size_t pix = (size_t)py * q.w + px;
    if (MODE == VR_COMPOSITE)
        reinterpret_cast<float4*>(q.out)[pix] = make_float4(acc.r, acc.g, acc.b, acc.A);
    else
        q.out[pix] = acc.m;
    return (unsigned)k;
}

// Kind of a textured request: (texel format, mode, more than one group).
__host__ __device__ constexpr int tex_kind(int format, int mode, bool multi)
{
    return (format * 3 + mode) * 2 + (multi ? 1 : 0);
}

// One switch over the kinds (uniform over the block: a tile belongs to one
// request); each case is the specialised march of one texel format and mode
// for a volume held in one layered texture.  (Volumes whose plain-format
// texture spans several layer groups go to their own launch with the
// run-time dispatched march: specialising them here as well makes the
// compiler merge the cases' code and spill.)
__device__ __forceinline__ unsigned tex_pixel_any(const BatchReq& q, const BatchTex& T,
                                                  const float4* __restrict__ lut, int px, int py)
{
    switch (tex_kind(T.format, q.mode, T.n_groups > 1)) {
#define VR_KIND(F, M) \
    case tex_kind(F, M, false): return tex_pixel<F, M, false>(q, T, lut, px, py);
#define VR_FORMAT(F) VR_KIND(F, VR_MIP) VR_KIND(F, VR_COMPOSITE) VR_KIND(F, VR_SUM)
        VR_FORMAT(VR_F32)
        VR_FORMAT(VR_F16)
        VR_FORMAT(VR_I8)
        VR_FORMAT(kF16Pair)
        VR_FORMAT(kI8Pair)
#undef VR_FORMAT
#undef VR_KIND
    default: return 0;
    }
}

// CLS (BatchClass): every request of the launch is of one class, so each
// kernel instance compiles one fetch path: bricks (run-time storage type),
// one layered texture (specialised per kind), several layer groups
// (run-time dispatched texture march).
template <int CLS>
__global__ void __launch_bounds__(kThreads, VR_BATCH_MIN_BLOCKS) batch_kernel(const __grid_constant__ BatchParams B,
                                                         unsigned* __restrict__ ws)
{
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
        const int tx = t % q.tiles_x, ty = t / q.tiles_x;
        const int px = tx * kTile + (warp & 1) * 8 + (lane & 7);
        const int py = ty * kTile + (warp >> 1) * 4 + (lane >> 3);
        unsigned count = 0;
        if (px < q.w && py < q.h) {
            if constexpr (CLS == kBatchTex) {
                count = tex_pixel_any(q, B.tex[q.tex_slot], s_lut, px, py);
            } else {
                const ray::Ray r = ray::setup_ray(q, q.cam, px, py, q.k_max);
                AccRT acc(q.mode);
                count = CLS == kBatchTexGroups
                            ? (unsigned)march_tex_rt(q, B.tex[q.tex_slot], s_lut, r, acc)
                            : (unsigned)march_bricks_rt(q, s_lut, r, acc);
                const size_t pix = (size_t)py * q.w + px;
                if (q.mode == VR_COMPOSITE)
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

cudaError_t launch_batch(const BatchParams& b, unsigned* ws, int grid, int cls, cudaStream_t s)
{
    // the counters start at zero for every launch (stream-ordered, capturable)
    cudaError_t e = cudaMemsetAsync(ws, 0, sizeof(unsigned) * (1 + b.n), s);
    if (e != cudaSuccess) return e;
    switch (cls) {
    case kBatchTex: batch_kernel<kBatchTex><<<grid, kThreads, 0, s>>>(b, ws); break;
    case kBatchTexGroups: batch_kernel<kBatchTexGroups><<<grid, kThreads, 0, s>>>(b, ws); break;
    default: batch_kernel<kBatchBricks><<<grid, kThreads, 0, s>>>(b, ws); break;
    }
    return cudaGetLastError();
}

int batch_blocks_per_sm(int cls)
{
    int n = 0;
    cudaError_t e =
        cls == kBatchTex
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<kBatchTex>, kThreads, 0)
        : cls == kBatchTexGroups
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<kBatchTexGroups>,
                                                            kThreads, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<kBatchBricks>,
                                                            kThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace vr
