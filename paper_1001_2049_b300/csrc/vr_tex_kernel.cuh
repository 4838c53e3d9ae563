// vr_tex_kernel.cuh -- the texture-gather ray-march kernel template and its
// launchers.  Instantiated once per texel format (vr_tex_<format>.cu) so the
// formats compile in parallel; vr_tex.cu dispatches between them.
//
// Same rendering as vr_march.cu (paper §3.1 process item 3; definition in
// include/vr.h).  The difference is where the eight corners of a cell come
// from: the cube is also held as layered 2-D textures (one layer per
// frequency plane z, block-linear in x and y), and one `tld4` (four-texel
// gather) returns the 2 x 2 corners of a cell in one plane.  A sample needs
// at most two gathers (planes z0 and z0 + 1) and no address arithmetic; the
// texture unit's 2-D tiling keeps the neighbouring rays of a warp on few
// cache lines whichever way the rays run.  The gathers return the stored
// texels unfiltered, so the interpolation (x, then y, then z, FP32) is the
// kernel's own and the results are those of the definition.
//
// The gathers of the next sample are issued before the current sample is
// interpolated, which hides the texture latency behind the arithmetic.
// With empty-space masks attached (SKIP, COMPOSITE), samples whose cell the
// clip makes transparent are not fetched (vr_ray.cuh, march_tex_win); with
// MIP bounds attached (SKIP, MIP, FP32) the march reads 8-bit upper-bound
// codes and fetches the FP32 corners only where a sample could raise the
// maximum (march_tex_bound).
#pragma once

#include <cuda_fp16.h>

#include "vr_internal.h"
#include "vr_ray.cuh"

namespace vr {
namespace tex {

// Launch shapes the autotuner chooses from: a block of BX x BY rays (one
// thread each), warps holding PX x PY packets of neighbouring rays, and the
// minimum number of resident blocks per SM the register budget must allow.
struct Shape {
    int bx, by, px, py, minb;
};
constexpr Shape kShapes[] = {
    {16, 16, 8, 4, 1}, {16, 16, 8, 4, 6}, {32, 8, 8, 4, 5}, {16, 16, 16, 2, 5},
    {16, 16, 4, 8, 5}, {8, 8, 8, 4, 16},
    {16, 8, 8, 4, 8}, {8, 16, 8, 4, 8}, {16, 16, 8, 4, 4},
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

template <int DT, int MODE, bool STACK, int CFG, bool SKIP>
__global__ void __launch_bounds__(kShapes[CFG].bx * kShapes[CFG].by, kShapes[CFG].minb)
    tex_kernel(const __grid_constant__ MarchParams P, const __grid_constant__ TexParams T)
{
    constexpr Shape S = kShapes[CFG];
    __shared__ float4 s_lut[VR_MAX_LUT];
    if (MODE == VR_COMPOSITE) {
        for (int i = threadIdx.x; i < P.n_lut; i += blockDim.x) s_lut[i] = P.lut[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int wpr = S.bx / S.px;                 // warps per block row
    const int px = blockIdx.x * S.bx + (warp % wpr) * S.px + (lane % S.px);
    const int py = blockIdx.y * S.by + (warp / wpr) * S.py + (lane / S.px);
    const int view = blockIdx.z;
    const bool valid = px < P.w && py < P.h;
    unsigned count = 0;
    if (valid) {
        const ray::Ray r = ray::setup_ray(P, P.cams[view], px, py, T.k_max);
        ray::Acc<MODE> acc;
        if constexpr (SKIP && MODE == VR_MIP)
            count = (unsigned)ray::march_tex_bound<STACK>(P, T, r, acc);
        else if constexpr (SKIP)
            count = (unsigned)ray::march_tex_win<DT, MODE, STACK>(P, T, s_lut, r, acc);
        else
            count = (unsigned)ray::march_tex<DT, MODE, STACK>(P, T, s_lut, r, acc);
        const size_t pix = ((size_t)view * P.h + py) * P.w + px;
        if (!ray::debug_ok(pix < (size_t)P.n_views * P.h * P.w, 1)) {
        } else if (MODE == VR_COMPOSITE)
            reinterpret_cast<float4*>(P.out)[pix] = make_float4(acc.r, acc.g, acc.b, acc.A);
        else
            P.out[pix] = acc.m;
    }
    if (P.samples) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, count);
        if (lane == 0 && tot) atomicAdd(P.samples, (unsigned long long)tot);
    }
}

template <int DT, int MODE, bool STACK, int CFG>
cudaError_t launch_c(const MarchParams& p, const TexParams& t, cudaStream_t s)
{
    // SKIP: COMPOSITE with empty-space masks (cells the clip makes
    // transparent are not fetched); MIP on FP32 storage with MIP bounds (the
    // march reads the 8-bit bound codes and fetches the FP32 corners only of
    // samples that could raise the maximum).  Passing over MIP samples by
    // their cells' corner maxima would not pay: on noise about a quarter of
    // the cells have a corner above a ray's running maximum, so nearly every
    // warp step would have a lane needing its sample.
    constexpr bool kCanSkip = MODE == VR_COMPOSITE || (MODE == VR_MIP && DT == VR_F32);
    constexpr Shape S = kShapes[CFG];
    dim3 grid((unsigned)((p.w + S.bx - 1) / S.bx), (unsigned)((p.h + S.by - 1) / S.by),
              (unsigned)p.n_views);
    const bool skip = MODE == VR_COMPOSITE ? p.mask != nullptr : t.bound != 0;
    if (kCanSkip && skip)
        tex_kernel<DT, MODE, STACK, CFG, kCanSkip><<<grid, S.bx * S.by, 0, s>>>(p, t);
    else
        tex_kernel<DT, MODE, STACK, CFG, false><<<grid, S.bx * S.by, 0, s>>>(p, t);
    return cudaGetLastError();
}

template <int DT, int MODE, bool STACK>
cudaError_t launch_m(const MarchParams& p, const TexParams& t, int cfg, cudaStream_t s)
{
    switch (cfg) {
    case 1: return launch_c<DT, MODE, STACK, 1>(p, t, s);
    case 2: return launch_c<DT, MODE, STACK, 2>(p, t, s);
    case 3: return launch_c<DT, MODE, STACK, 3>(p, t, s);
    case 4: return launch_c<DT, MODE, STACK, 4>(p, t, s);
    case 5: return launch_c<DT, MODE, STACK, 5>(p, t, s);
    case 6: return launch_c<DT, MODE, STACK, 6>(p, t, s);
    case 7: return launch_c<DT, MODE, STACK, 7>(p, t, s);
    case 8: return launch_c<DT, MODE, STACK, 8>(p, t, s);
    default: return launch_c<DT, MODE, STACK, 0>(p, t, s);
    }
}
static_assert(kNumShapes == 9, "launch_m lists every shape");

template <int DT, int MODE>
cudaError_t launch_t(const MarchParams& p, const TexParams& t, int cfg, cudaStream_t s)
{
    return t.stack_shift > 0 ? launch_m<DT, MODE, true>(p, t, cfg, s)
                             : launch_m<DT, MODE, false>(p, t, cfg, s);
}

template <int DT>
cudaError_t launch_dt(const MarchParams& p, const TexParams& t, int mode, int cfg,
                      cudaStream_t s)
{
    switch (mode) {
    case VR_MIP: return launch_t<DT, VR_MIP>(p, t, cfg, s);
    case VR_COMPOSITE: return launch_t<DT, VR_COMPOSITE>(p, t, cfg, s);
    default: return launch_t<DT, VR_SUM>(p, t, cfg, s);
    }
}

// One part of a larger cube (vr_render_part): each ray of the whole cube
// whose direction matches the sweep continues from the state in `out` with
// the samples of the part's cells (the same samples, in the same order, as
// the one-pass render takes there), then writes the state back.
// MASKED (COMPOSITE with the part's empty-space masks): 16 x 8 blocks at 64
// registers, the shape at which the masked march ran fastest; otherwise
// 16 x 16 blocks at up to 51 registers (five blocks per SM).  Warps hold
// 8 x 4 packets either way.
template <int DT, int MODE, bool STACK, bool MASKED>
__global__ void __launch_bounds__(MASKED ? 128 : 256, MASKED ? 8 : 5)
    part_kernel(const __grid_constant__ MarchParams P, const __grid_constant__ TexParams T)
{
    constexpr int kRowsY = MASKED ? 8 : 16;
    __shared__ float4 s_lut[VR_MAX_LUT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int px = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int py = blockIdx.y * kRowsY + (warp >> 1) * 4 + (lane >> 3);
    const int view = blockIdx.z;
    // the ray, its state and its samples in this part (most rays of a view
    // cross a few parts only: a test of its first and last samples' cells
    // spares the others the bisection)
    ray::Ray r;
    ray::Acc<MODE> acc;
    size_t pix = 0;
    int k0 = 0, k1 = 0;
    if (px < P.w && py < P.h) {
        r = ray::setup_ray(P, P.cams[view], px, py, T.k_max);
        // sweep 0: every ray (a partial image rendered on its own)
        const bool mine = P.sweep == 0 || (P.sweep > 0 ? r.dz >= 0.0f : r.dz < 0.0f);
        if (r.K > 0 && mine && ray::may_cross_part(P, r)) {
            pix = ((size_t)view * P.h + py) * P.w + px;
            bool done = false;
            if (MODE == VR_COMPOSITE) {
                const float4 c = reinterpret_cast<const float4*>(P.out)[pix];
                acc.r = c.x;
                acc.g = c.y;
                acc.b = c.z;
                acc.A = c.w;
                done = acc.A >= P.term_alpha;          // the ray stopped in an earlier part
            } else {
                acc.m = P.out[pix];
            }
            if (!done) ray::part_range(P, r, k0, k1);
        }
    }
    // a ray without samples here keeps its state (nothing to write); blocks
    // whose rays all have none leave before staging the table
    const bool work = k0 < k1;
    if (!__syncthreads_or(work)) return;
    if (MODE == VR_COMPOSITE) {
        for (int i = threadIdx.x; i < P.n_lut; i += blockDim.x) s_lut[i] = P.lut[i];
        __syncthreads();
    }
    unsigned count = 0;
    if (work) {
        if constexpr (MODE == VR_MIP && DT == VR_F32) {
            // with MIP bounds (block-uniform), as the one-pass render
            count = T.bound ? (unsigned)ray::march_part_bound<STACK>(P, T, r, acc, k0, k1)
                            : (unsigned)ray::march_part<DT, MODE, STACK>(P, T, s_lut, r,
                                                                         acc, k0, k1);
        } else if constexpr (MODE == VR_COMPOSITE && MASKED) {
            // with empty-space masks, as the one-pass render
            count = (unsigned)ray::march_win<DT, VR_COMPOSITE, STACK, true>(P, T, s_lut, r,
                                                                             acc, k0, k1);
        } else {
            count = (unsigned)ray::march_part<DT, MODE, STACK>(P, T, s_lut, r, acc, k0,
                                                              k1);
        }
        if (!ray::debug_ok(pix < (size_t)P.n_views * P.h * P.w, 1)) {
        } else if (MODE == VR_COMPOSITE)
            reinterpret_cast<float4*>(P.out)[pix] =
                make_float4(acc.r, acc.g, acc.b, acc.A);
        else
            P.out[pix] = acc.m;
    }
    if (P.samples) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, count);
        if (lane == 0 && tot) atomicAdd(P.samples, (unsigned long long)tot);
    }
}

template <int DT>
cudaError_t launch_part_dt(const MarchParams& p, const TexParams& t, int mode, cudaStream_t s)
{
    const dim3 grid((unsigned)((p.w + 15) / 16), (unsigned)((p.h + 15) / 16),
                    (unsigned)p.n_views);
    const bool st = t.stack_shift > 0;
    switch (mode) {
    case VR_MIP:
        st ? part_kernel<DT, VR_MIP, true, false><<<grid, 256, 0, s>>>(p, t)
           : part_kernel<DT, VR_MIP, false, false><<<grid, 256, 0, s>>>(p, t);
        break;
    case VR_COMPOSITE:
        if (p.mask) {
            const dim3 g8((unsigned)((p.w + 15) / 16), (unsigned)((p.h + 7) / 8),
                          (unsigned)p.n_views);
            st ? part_kernel<DT, VR_COMPOSITE, true, true><<<g8, 128, 0, s>>>(p, t)
               : part_kernel<DT, VR_COMPOSITE, false, true><<<g8, 128, 0, s>>>(p, t);
        } else {
            st ? part_kernel<DT, VR_COMPOSITE, true, false><<<grid, 256, 0, s>>>(p, t)
               : part_kernel<DT, VR_COMPOSITE, false, false><<<grid, 256, 0, s>>>(p, t);
        }
        break;
    default:
        st ? part_kernel<DT, VR_SUM, true, false><<<grid, 256, 0, s>>>(p, t)
           : part_kernel<DT, VR_SUM, false, false><<<grid, 256, 0, s>>>(p, t);
        break;
    }
    return cudaGetLastError();
}

}  // namespace tex
}  // namespace vr
