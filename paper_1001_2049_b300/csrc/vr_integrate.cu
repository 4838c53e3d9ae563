// vr_integrate.cu -- scene integration: the partial images of sub-cubes
// rendered independently combined into one image per view.
//
// The paper's pipeline renders each sub-cube into an image and combines the
// images (§3.1 items 4, 5; its "scene integration" sentence is garbled and
// read here as combining the partial images by the compositing operator in
// visibility order).  For a ray the visibility order of z-slab sub-cubes is
// ascending z when it goes up (or is level) and descending when it goes
// down, the direction decided exactly as the part kernel decides it
// (ray_dz_raw).  Per pixel, front to back:
//   COMPOSITE  C += (1 - A) C_i, A += (1 - A) A_i   (premultiplied RGBA)
//   MIP        max of the partial maxima
//   SUM        sum of the partial sums
// One thread per pixel; the partial images are read once, coalesced (16 B
// per composite pixel and part): HBM-bound, parts x image bytes read plus
// one image written.
#include <algorithm>

#include "vr_internal.h"
#include "vr_ray.cuh"

namespace vr {
namespace {

template <int MODE>
__global__ void __launch_bounds__(256) integrate_kernel(const __grid_constant__ IntegrateParams P)
{
    const size_t per_view = (size_t)P.w * P.h;
    const size_t n = per_view * P.n_views;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        // 64-bit until the coordinates: one view may hold more than 2^31 pixels
        const int view = (int)(i / per_view);
        const size_t rem = i - (size_t)view * per_view;
        const int py = (int)(rem / (size_t)P.w), px = (int)(rem - (size_t)py * P.w);
        const bool up = ray::ray_dz_raw(P.cams[view], P.w, P.h, px, py) >= 0.0f;
        if constexpr (MODE == VR_COMPOSITE) {
            const float4* src = reinterpret_cast<const float4*>(P.partials);
            float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            for (int j = 0; j < P.n_parts; ++j) {
                const int part = up ? j : P.n_parts - 1 - j;
                const size_t at = (size_t)part * P.part_stride + i;
                if (!ray::debug_ok(at < (size_t)P.n_parts * P.part_stride, 4)) continue;
                const float4 c = src[at];
                const float T = 1.0f - acc.w;
                acc.x = fmaf(T, c.x, acc.x);
                acc.y = fmaf(T, c.y, acc.y);
                acc.z = fmaf(T, c.z, acc.z);
                acc.w = fmaf(T, c.w, acc.w);
            }
            reinterpret_cast<float4*>(P.out)[i] = acc;
        } else {
            float acc = MODE == VR_MIP ? -INFINITY : 0.0f;
            for (int j = 0; j < P.n_parts; ++j) {
                const int part = up ? j : P.n_parts - 1 - j;
                const float v = P.partials[(size_t)part * P.part_stride + i];
                acc = MODE == VR_MIP ? fmaxf(acc, v) : acc + v;
            }
            P.out[i] = acc;
        }
    }
}

}  // namespace

cudaError_t launch_integrate(const IntegrateParams& p, int mode, cudaStream_t s)
{
    const size_t n = (size_t)p.w * p.h * p.n_views;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t want = (n + 255) / 256;
    const unsigned grid = (unsigned)std::min<size_t>(want, (size_t)sms * 8);
    switch (mode) {
    case VR_COMPOSITE: integrate_kernel<VR_COMPOSITE><<<grid, 256, 0, s>>>(p); break;
    case VR_MIP: integrate_kernel<VR_MIP><<<grid, 256, 0, s>>>(p); break;
    default: integrate_kernel<VR_SUM><<<grid, 256, 0, s>>>(p); break;
    }
    return cudaGetLastError();
}

// the checked build's device word of this translation unit
VR_DEBUG_ACCESSOR(debug_flags_integrate)

}  // namespace vr
