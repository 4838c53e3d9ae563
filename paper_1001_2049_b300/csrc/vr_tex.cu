// vr_tex.cu -- texture storage: the fill kernels that copy the bricks into
// layered textures, the texel-format dispatch of the texture-gather march
// (the kernel itself: vr_tex_kernel.cuh) and the launch-shape table.
//
// Layers: a layered texture holds at most kMaxLayers layers, so deeper cubes
// stack 2^shift planes per layer (see write_slice_row).
#include <algorithm>
#include <type_traits>

#include <cuda_fp16.h>

#include "vr_internal.h"
#include "vr_tex_kernel.cuh"

namespace vr {
namespace {

// Slice z of the texture (see vr_ray.cuh for what the slices hold) is 2-D
// sub-slice z & (2^shift - 1) of layer z >> shift.  Unstacked (shift 0) a slice
// is the ny rows of data; stacked, a slice spans `pitch` = ny + 2 rows: a
// copy of data row 0, the ny data rows, a copy of data row ny - 1, so a
// gather one row outside the data reads the edge row exactly as the
// texture's clamp addressing does for an unstacked layer.
template <typename W>
__device__ __forceinline__ void write_slice_row(cudaSurfaceObject_t surf, W v, int x, int y,
                                                int z, int ny, int shift, int pitch)
{
    const int layer = z >> shift;
    if (shift == 0) {
        surf2DLayeredwrite(v, surf, x * (int)sizeof(W), y, layer);
        return;
    }
    const int base = (z & ((1 << shift) - 1)) * pitch + 1;
    surf2DLayeredwrite(v, surf, x * (int)sizeof(W), base + y, layer);
    if (y == 0) surf2DLayeredwrite(v, surf, x * (int)sizeof(W), base - 1, layer);
    if (y == ny - 1) surf2DLayeredwrite(v, surf, x * (int)sizeof(W), base + ny, layer);
}

// *vmax = max(*vmax, the largest m of the block's 256 threads); one atomic per
// block (the bit patterns of values >= 0 order as integers).  Every thread of
// the block calls it.
__device__ __forceinline__ void raise_max(float m, float* vmax)
{
    __shared__ float warp_max[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, warp_max[w]);
        atomicMax(reinterpret_cast<int*>(vmax), __float_as_int(m));
    }
}

// Plain formats: slices [s0, s1) of the texture; slice s holds plane s - 1,
// slices 0 and nz + 1 repeat the edge planes.
template <typename T>
__global__ void __launch_bounds__(256) fill_kernel(const T* __restrict__ bricks, VolumeGeom g,
                                                   cudaSurfaceObject_t surf, int s0, int s1,
                                                   int shift, int pitch)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= g.nx || y >= g.ny) return;
    for (int sl = s0 + blockIdx.z; sl < s1; sl += gridDim.z) {
        const int z = min(max(sl - 1, 0), g.nz - 1);
        const size_t brick = ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx +
                             (x >> kBrickShift);
        const T v = bricks[brick * kBrickVoxels + ((z & 31) << 10) + ((y & 31) << 5) + (x & 31)];
        write_slice_row(surf, v, x, y, sl, g.ny, shift, pitch);
    }
}

// A float rounded toward +infinity to bfloat16 (its upper 16 bits): never
// below the value; truncating the low bits raises a negative value, so only
// positive values with low bits set move up one bfloat16 step (the largest
// finite value to +inf).  NaN stays NaN (a NaN bound is never below a
// running maximum, so its samples are always evaluated).
__device__ __forceinline__ unsigned bf16_up(float v)
{
    const unsigned b = __float_as_uint(v);
    if (v != v) return 0x7fc0u;
    const unsigned hi = b >> 16;
    return ((b & 0xffffu) != 0u && !(b >> 31)) ? hi + 1u : hi;
}

// The MIP-bound texel of cell slice sl at (x, y): the voxels of planes sl - 1
// and sl (clamped to the cube), each rounded up to bfloat16, packed low =
// plane sl - 1 (the pair layout of vr_ray.cuh); m is raised to their
// largest |value| (NaN ignored).  The march reads the whole texel as the
// upper plane's bound, the low half adding less than one bfloat16 step of
// magnitude: so a negative upper bound is stored one step further up (a
// bound of magnitude at most one step becomes +0).
__device__ __forceinline__ unsigned bound_texel(const float* __restrict__ bricks,
                                                const VolumeGeom& g, int x, int y, int sl,
                                                float& m)
{
    const size_t row = ((size_t)(y >> kBrickShift) * g.nbx + (x >> kBrickShift)) * kBrickVoxels +
                       ((y & 31) << 5) + (x & 31);
    const size_t slab = (size_t)g.nbx * g.nby * kBrickVoxels;
    const int za = min(max(sl - 1, 0), g.nz - 1), zb = min(sl, g.nz - 1);
    const float lo = bricks[(size_t)(za >> kBrickShift) * slab + row + ((za & 31) << 10)];
    const float hi = bricks[(size_t)(zb >> kBrickShift) * slab + row + ((zb & 31) << 10)];
    m = fmaxf(m, fmaxf(fabsf(lo), fabsf(hi)));
    unsigned h = bf16_up(hi);
    if (h & 0x8000u) h = (h & 0x7fffu) <= 1u ? 0u : h - 1u;
    return bf16_up(lo) | (h << 16);
}

// MIP bounds: cell slices [s0, s1) (slice s holds planes s - 1 and s, s in
// [0, nz]) through a surface, stacked as the FP32 texture's slices.  Also
// raises *vmax to the largest |voxel| read: |voxel| >= 0, so its bit pattern
// orders as an integer.
__global__ void __launch_bounds__(256) fill_bound_kernel(const float* __restrict__ bricks,
                                                         VolumeGeom g, cudaSurfaceObject_t surf,
                                                         int s0, int s1, int shift, int pitch,
                                                         float* __restrict__ vmax)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    float m = 0.0f;
    if (x < g.nx && y < g.ny) {
        for (int sl = s0 + blockIdx.z; sl < s1; sl += gridDim.z)
            write_slice_row(surf, bound_texel(bricks, g, x, y, sl, m), x, y, sl, g.ny, shift,
                            pitch);
    }
    raise_max(m, vmax);
}

// fill_bound_kernel's slices written linearly: slice s0 + j at dst + j nx ny,
// x fastest (for a copy into an unstacked bound texture).
__global__ void __launch_bounds__(256) fill_bound_linear_kernel(
    const float* __restrict__ bricks, VolumeGeom g, unsigned* __restrict__ dst, int s0, int s1,
    float* __restrict__ vmax)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    float m = 0.0f;
    if (x < g.nx && y < g.ny) {
        for (int sl = s0 + blockIdx.z; sl < s1; sl += gridDim.z)
            dst[((size_t)(sl - s0) * g.ny + y) * g.nx + x] = bound_texel(bricks, g, x, y, sl, m);
    }
    raise_max(m, vmax);
}

// Pair formats: slices [s0, s1); slice s holds the voxels of planes s - 1 and
// s (clamped to the cube) packed in one texel, low bits plane s - 1.
template <typename T, typename W>
__global__ void __launch_bounds__(256) fill_pair_kernel(const T* __restrict__ bricks, VolumeGeom g,
                                                        cudaSurfaceObject_t surf, int s0, int s1,
                                                        int shift, int pitch)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= g.nx || y >= g.ny) return;
    const size_t row = ((size_t)(y >> kBrickShift) * g.nbx + (x >> kBrickShift)) * kBrickVoxels +
                       ((y & 31) << 5) + (x & 31);
    const size_t slab = (size_t)g.nbx * g.nby * kBrickVoxels;
    for (int sl = s0 + blockIdx.z; sl < s1; sl += gridDim.z) {
        const int za = min(max(sl - 1, 0), g.nz - 1), zb = min(sl, g.nz - 1);
        const T lo = bricks[(size_t)(za >> kBrickShift) * slab + row + ((za & 31) << 10)];
        const T hi = bricks[(size_t)(zb >> kBrickShift) * slab + row + ((zb & 31) << 10)];
        const W packed = (W)((W)(unsigned)(typename std::make_unsigned<T>::type)lo |
                             ((W)(unsigned)(typename std::make_unsigned<T>::type)hi
                              << (8 * sizeof(T))));
        write_slice_row(surf, packed, x, y, sl, g.ny, shift, pitch);
    }
}

}  // namespace

cudaError_t launch_tex(const MarchParams& p, const TexParams& t, int format, int mode, int cfg,
                       cudaStream_t s)
{
    if (cfg < 0 || cfg >= tex::kNumShapes) cfg = 0;
    switch (format) {
    case VR_F32: return launch_tex_f32(p, t, mode, cfg, s);
    case VR_F16: return launch_tex_f16(p, t, mode, cfg, s);
    case kF16Pair: return launch_tex_f16pair(p, t, mode, cfg, s);
    case kI8Pair: return launch_tex_i8pair(p, t, mode, cfg, s);
    default: return launch_tex_i8(p, t, mode, cfg, s);
    }
}

cudaError_t launch_part(const MarchParams& p, const TexParams& t, int format, int mode,
                        cudaStream_t s)
{
    switch (format) {
    case VR_F32: return launch_part_f32(p, t, mode, s);
    case VR_F16: return launch_part_f16(p, t, mode, s);
    case kF16Pair: return launch_part_f16pair(p, t, mode, s);
    case kI8Pair: return launch_part_i8pair(p, t, mode, s);
    default: return launch_part_i8(p, t, mode, s);
    }
}

namespace {
__global__ void __launch_bounds__(256) dec_kernel(const float* __restrict__ scale,
                                                  const float* __restrict__ offset, int nz,
                                                  bool pair, void* __restrict__ out, int n)
{
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= n) return;
    const int z0 = min(max(sl - 1, 0), nz - 1), z1 = min(sl, nz - 1);
    if (pair)
        static_cast<float4*>(out)[sl] = make_float4(scale[z0], offset[z0], scale[z1], offset[z1]);
    else
        static_cast<float2*>(out)[sl] = make_float2(scale[z0], offset[z0]);
}

__global__ void __launch_bounds__(256) init_kernel(float* __restrict__ out, size_t n, float v)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = v;
}
}  // namespace

cudaError_t fill_decode_records(const Volume& v, cudaStream_t s)
{
    const bool pair = v.tex_format == kI8Pair;
    const int n = pair ? v.g.nz + 1 : v.g.nz + 2;
    dec_kernel<<<(n + 255) / 256, 256, 0, s>>>(v.scale, v.offset, v.g.nz, pair, v.dec, n);
    return cudaGetLastError();
}

cudaError_t launch_render_init(float* out, size_t n_pixels, int mode, cudaStream_t s)
{
    const size_t n = n_pixels * (mode == VR_COMPOSITE ? 4 : 1);
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 148 * 32);
    init_kernel<<<blocks, 256, 0, s>>>(out, n, mode == VR_MIP ? -INFINITY : 0.0f);
    return cudaGetLastError();
}

int tex_shape_count() { return tex::kNumShapes; }

void tex_shape(int cfg, int* bx, int* by, int* px, int* py, int* minb)
{
    const tex::Shape& sh = tex::kShapes[cfg];
    *bx = sh.bx;
    *by = sh.by;
    *px = sh.px;
    *py = sh.py;
    *minb = sh.minb;
}

// The bound fills' grid: 32 x 8 voxel rows per block, at most 32 blocks along
// the slices (each block then walks several slices), so that the maximum
// takes a few thousand atomics on one word rather than one per warp row.
static dim3 bound_grid(const Volume& v, int z0, int z1)
{
    return dim3((unsigned)((v.g.nx + 31) / 32), (unsigned)((v.g.ny + 7) / 8),
                (unsigned)std::min(z1 - z0, 32));
}

cudaError_t fill_bounds(const Volume& v, cudaSurfaceObject_t surf, int z0, int z1, float* vmax,
                        cudaStream_t s)
{
    if (z1 <= z0) return cudaSuccess;
    const dim3 grid = bound_grid(v, z0, z1);
    fill_bound_kernel<<<grid, 256, 0, s>>>((const float*)v.bricks, v.g, surf, z0, z1,
                                           v.stack_shift, v.stack_pitch, vmax);
    return cudaGetLastError();
}

cudaError_t fill_bounds_linear(const Volume& v, unsigned* dst, int z0, int z1, float* vmax,
                               cudaStream_t s)
{
    if (z1 <= z0) return cudaSuccess;
    const dim3 grid = bound_grid(v, z0, z1);
    fill_bound_linear_kernel<<<grid, 256, 0, s>>>((const float*)v.bricks, v.g, dst, z0, z1, vmax);
    return cudaGetLastError();
}

cudaError_t fill_texture(const Volume& v, cudaSurfaceObject_t surf, int z0, int z1, cudaStream_t s)
{
    if (z1 <= z0) return cudaSuccess;
    dim3 grid((unsigned)((v.g.nx + 31) / 32), (unsigned)((v.g.ny + 7) / 8),
              (unsigned)((z1 - z0) < 1024 ? (z1 - z0) : 1024));
    const int sh = v.stack_shift, pt = v.stack_pitch;
    if (v.tex_format == kF16Pair) {
        fill_pair_kernel<unsigned short, unsigned int><<<grid, 256, 0, s>>>(
            (const unsigned short*)v.bricks, v.g, surf, z0, z1, sh, pt);
        return cudaGetLastError();
    }
    if (v.tex_format == kI8Pair) {
        fill_pair_kernel<signed char, unsigned short><<<grid, 256, 0, s>>>(
            (const signed char*)v.bricks, v.g, surf, z0, z1, sh, pt);
        return cudaGetLastError();
    }
    switch (v.dtype) {
    case VR_F32:
        fill_kernel<float><<<grid, 256, 0, s>>>((const float*)v.bricks, v.g, surf, z0, z1, sh, pt);
        break;
    case VR_F16:   // binary16 bit patterns moved as 16-bit words
        fill_kernel<unsigned short><<<grid, 256, 0, s>>>((const unsigned short*)v.bricks, v.g,
                                                         surf, z0, z1, sh, pt);
        break;
    default:
        fill_kernel<signed char><<<grid, 256, 0, s>>>((const signed char*)v.bricks, v.g, surf, z0,
                                                      z1, sh, pt);
        break;
    }
    return cudaGetLastError();
}

}  // namespace vr
