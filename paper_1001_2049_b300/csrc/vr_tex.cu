// vr_tex.cu -- the texture-gather ray-march kernel (the render hot path when a
// volume has texture storage attached).
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
//
// Layers: a layered texture holds at most kMaxLayers planes, so the cube is
// split into groups of planes [g*(L-1), g*(L-1) + L) that overlap by one
// plane; the plane pair (z0, z0 + 1) always lies in one group.
#include <type_traits>

#include <cuda_fp16.h>

#include "vr_internal.h"
#include "vr_ray.cuh"

namespace vr {
namespace {

// Launch shapes the autotuner chooses from: a block of BX x BY rays (one
// thread each), warps holding PX x PY packets of neighbouring rays, and the
// minimum number of resident blocks per SM the register budget must allow.
struct Shape {
    int bx, by, px, py, minb;
};
constexpr Shape kShapes[] = {
    {16, 16, 8, 4, 1}, {16, 16, 8, 4, 6}, {32, 8, 8, 4, 5}, {16, 16, 16, 2, 5},
    {16, 16, 4, 8, 5}, {8, 8, 8, 4, 16},
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

template <int DT, int MODE, bool MULTI, int CFG>
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
        count = (unsigned)ray::march_tex<DT, MODE, MULTI>(P, T, s_lut, r, acc);
        const size_t pix = ((size_t)view * P.h + py) * P.w + px;
        if (MODE == VR_COMPOSITE)
            reinterpret_cast<float4*>(P.out)[pix] = make_float4(acc.r, acc.g, acc.b, acc.A);
        else
            P.out[pix] = acc.m;
    }
    if (P.samples) {
        const unsigned tot = __reduce_add_sync(0xffffffffu, count);
        if (lane == 0 && tot) atomicAdd(P.samples, (unsigned long long)tot);
    }
}

template <int DT, int MODE, bool MULTI, int CFG>
cudaError_t launch_c(const MarchParams& p, const TexParams& t, cudaStream_t s)
{
    constexpr Shape S = kShapes[CFG];
    dim3 grid((unsigned)((p.w + S.bx - 1) / S.bx), (unsigned)((p.h + S.by - 1) / S.by),
              (unsigned)p.n_views);
    tex_kernel<DT, MODE, MULTI, CFG><<<grid, S.bx * S.by, 0, s>>>(p, t);
    return cudaGetLastError();
}

template <int DT, int MODE, bool MULTI>
cudaError_t launch_m(const MarchParams& p, const TexParams& t, int cfg, cudaStream_t s)
{
    switch (cfg) {
    case 1: return launch_c<DT, MODE, MULTI, 1>(p, t, s);
    case 2: return launch_c<DT, MODE, MULTI, 2>(p, t, s);
    case 3: return launch_c<DT, MODE, MULTI, 3>(p, t, s);
    case 4: return launch_c<DT, MODE, MULTI, 4>(p, t, s);
    case 5: return launch_c<DT, MODE, MULTI, 5>(p, t, s);
    default: return launch_c<DT, MODE, MULTI, 0>(p, t, s);
    }
}
static_assert(kNumShapes == 6, "launch_m lists every shape");

template <int DT, int MODE>
cudaError_t launch_t(const MarchParams& p, const TexParams& t, int cfg, cudaStream_t s)
{
    return t.n_groups > 1 ? launch_m<DT, MODE, true>(p, t, cfg, s)
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

// Copy planes [z0, z1) from the bricks into texture group g (surface writes).
template <typename T>
__global__ void __launch_bounds__(256) fill_kernel(const T* __restrict__ bricks, VolumeGeom g,
                                                   cudaSurfaceObject_t surf, int layer0, int z0,
                                                   int z1)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= g.nx || y >= g.ny) return;
    for (int z = z0 + blockIdx.z; z < z1; z += gridDim.z) {
        const size_t brick = ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx +
                             (x >> kBrickShift);
        const T v = bricks[brick * kBrickVoxels + ((z & 31) << 10) + ((y & 31) << 5) + (x & 31)];
        surf2DLayeredwrite(v, surf, x * (int)sizeof(T), y, z - layer0);
    }
}

// Pair formats: layer l of the group holds cell plane c = first + l, i.e. the
// voxels of planes c and c + 1 packed into one texel (low bits: plane c).
template <typename T, typename W>
__global__ void __launch_bounds__(256) fill_pair_kernel(const T* __restrict__ bricks, VolumeGeom g,
                                                        cudaSurfaceObject_t surf, int first,
                                                        int c0, int c1)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= g.nx || y >= g.ny) return;
    const size_t row = ((size_t)(y >> kBrickShift) * g.nbx + (x >> kBrickShift)) * kBrickVoxels +
                       ((y & 31) << 5) + (x & 31);
    const size_t slab = (size_t)g.nbx * g.nby * kBrickVoxels;
    for (int c = c0 + blockIdx.z; c < c1; c += gridDim.z) {
        const T lo = bricks[(size_t)(c >> kBrickShift) * slab + row + ((c & 31) << 10)];
        const int c_ = c + 1;
        const T hi = bricks[(size_t)(c_ >> kBrickShift) * slab + row + ((c_ & 31) << 10)];
        const W packed = (W)((W)(unsigned)(typename std::make_unsigned<T>::type)lo |
                             ((W)(unsigned)(typename std::make_unsigned<T>::type)hi
                              << (8 * sizeof(T))));
        surf2DLayeredwrite(packed, surf, x * (int)sizeof(W), y, c - first);
    }
}

}  // namespace

cudaError_t launch_tex(const MarchParams& p, const TexParams& t, int format, int mode, int cfg,
                       cudaStream_t s)
{
    if (cfg < 0 || cfg >= kNumShapes) cfg = 0;
    switch (format) {
    case VR_F32: return launch_dt<VR_F32>(p, t, mode, cfg, s);
    case VR_F16: return launch_dt<VR_F16>(p, t, mode, cfg, s);
    case kF16Pair: return launch_dt<kF16Pair>(p, t, mode, cfg, s);
    case kI8Pair: return launch_dt<kI8Pair>(p, t, mode, cfg, s);
    default: return launch_dt<VR_I8>(p, t, mode, cfg, s);
    }
}

int tex_shape_count() { return kNumShapes; }

void tex_shape(int cfg, int* bx, int* by, int* px, int* py, int* minb)
{
    const Shape& sh = kShapes[cfg];
    *bx = sh.bx;
    *by = sh.by;
    *px = sh.px;
    *py = sh.py;
    *minb = sh.minb;
}

cudaError_t fill_texture_group(const Volume& v, cudaSurfaceObject_t surf, int layer0, int z0,
                               int z1, cudaStream_t s)
{
    dim3 grid((unsigned)((v.g.nx + 31) / 32), (unsigned)((v.g.ny + 7) / 8),
              (unsigned)((z1 - z0) < 1024 ? (z1 - z0) : 1024));
    if (v.tex_format == kF16Pair) {
        fill_pair_kernel<unsigned short, unsigned int><<<grid, 256, 0, s>>>(
            (const unsigned short*)v.bricks, v.g, surf, layer0, z0, z1);
        return cudaGetLastError();
    }
    if (v.tex_format == kI8Pair) {
        fill_pair_kernel<signed char, unsigned short><<<grid, 256, 0, s>>>(
            (const signed char*)v.bricks, v.g, surf, layer0, z0, z1);
        return cudaGetLastError();
    }
    switch (v.dtype) {
    case VR_F32:
        fill_kernel<float><<<grid, 256, 0, s>>>((const float*)v.bricks, v.g, surf, layer0, z0, z1);
        break;
    case VR_F16:   // binary16 bit patterns moved as 16-bit words
        fill_kernel<unsigned short><<<grid, 256, 0, s>>>((const unsigned short*)v.bricks, v.g,
                                                         surf, layer0, z0, z1);
        break;
    default:
        fill_kernel<signed char><<<grid, 256, 0, s>>>((const signed char*)v.bricks, v.g, surf,
                                                      layer0, z0, z1);
        break;
    }
    return cudaGetLastError();
}

}  // namespace vr
