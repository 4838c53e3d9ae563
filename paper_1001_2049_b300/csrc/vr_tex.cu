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

// ---- MIP bounds: 8-bit upper-bound codes (BoundScale) ----

// Order-preserving bit pattern of a float: unsigned comparison of the
// patterns orders the values (negative values have every bit flipped,
// non-negative ones the sign bit set).
__device__ __forceinline__ unsigned ordered_bits(float v)
{
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float from_ordered(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Address of voxel (x, y, z) in the FP32 bricks.
__device__ __forceinline__ size_t voxel_index(const VolumeGeom& g, int x, int y, int z)
{
    return ((size_t)((z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx +
            (x >> kBrickShift)) * kBrickVoxels +
           ((z & 31) << 10) + ((y & 31) << 5) + (x & 31);
}

__global__ void bound_reset_kernel(BoundScale* __restrict__ b)
{
    b->lo = 0xffffffffu;
    b->hi = 0u;
    b->inf = 0u;
}

// The smallest and largest finite voxel of the cube (each thread a column of
// voxels along z, one pair of atomics per block), and whether a voxel is +inf.
__global__ void __launch_bounds__(256) bound_range_kernel(const float* __restrict__ bricks,
                                                          VolumeGeom g,
                                                          BoundScale* __restrict__ b)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    unsigned lo = 0xffffffffu, hi = 0u, inf = 0u;
    if (x < g.nx && y < g.ny) {
        for (int z = blockIdx.z; z < g.nz; z += gridDim.z) {
            const float v = bricks[voxel_index(g, x, y, z)];
            if (isfinite(v)) {
                const unsigned k = ordered_bits(v);
                lo = min(lo, k);
                hi = max(hi, k);
            } else if (v > 0.0f) {
                inf = 1u;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        inf |= __shfl_xor_sync(0xffffffffu, inf, o);
    }
    __shared__ unsigned s_lo[8], s_hi[8], s_inf[8];
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
        s_inf[threadIdx.x >> 5] = inf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            lo = min(lo, s_lo[w]);
            hi = max(hi, s_hi[w]);
            inf |= s_inf[w];
        }
        atomicMin(&b->lo, lo);
        atomicMax(&b->hi, hi);
        if (inf) atomicOr(&b->inf, 1u);
    }
}

// The code scale from the cube's range [lo, hi]: L = lo, delta = (hi - lo) /
// 254 rounded up (so 255 delta exceeds the range by more than the rounding
// of the codes' test below), and the constants of the march's limit
// (vr_ray.cuh, bound_limit): le = L + e rounded up, where e = max(2^-19
// max|voxel|, 2^-126) covers the float rounding of a sample's own trilinear
// interpolation (at most 9 * 2^-24 of its largest |corner|, subnormal
// rounding included), and inv_q = 1 / (delta 2^15) rounded down.  Any
// non-finite step (no finite voxel, a +inf voxel, a range or scale that
// overflows) leaves le = +inf: then no sample is ever skipped.
__global__ void bound_finish_kernel(BoundScale* __restrict__ b)
{
    const bool any = b->lo <= b->hi;
    const float lo = any ? from_ordered(b->lo) : 0.0f, hi = any ? from_ordered(b->hi) : 0.0f;
    float delta = __fdiv_ru(__fsub_ru(hi, lo), 254.0f);
    delta = fmaxf(delta, 0x1p-126f);
    const float inv_q = __frcp_rd(delta * 32768.0f);
    const float vlim = fmaxf(fabsf(lo), fabsf(hi));
    const float le = __fadd_ru(lo, fmaxf(vlim * 0x1p-19f, 0x1p-126f));
    const bool ok = any && !b->inf && isfinite(delta) && isfinite(le) && inv_q > 0.0f &&
                    isfinite(inv_q);
    b->L = lo;
    b->delta = ok ? delta : 1.0f;
    b->inv_q = ok ? inv_q : 0.0f;
    b->le = ok ? le : INFINITY;
    b->vlim = vlim;
}

// The code of voxel v: a c in [0, 255] with L + c delta >= v in exact
// arithmetic -- checked with r = v - L rounded up and c delta rounded down,
// c * delta >= r, which implies it.  NaN and -inf take 0 (a sample with such
// a corner is NaN or -inf and never raises a maximum), values at or below L
// too.  A voxel the scale cannot cover (+inf, |v| beyond the magnitude le's
// rounding term was derived from, or no code reaching it) sets `off`:
// skipping must then be turned off.
__device__ __forceinline__ unsigned bound_code(float v, const BoundScale& b, bool& off)
{
    if (v != v || v == -INFINITY) return 0u;
    if (!(fabsf(v) <= b.vlim)) {          // beyond the range le covers (+inf included)
        off = true;
        return 255u;
    }
    if (!(v > b.L)) return 0u;
    const float r = __fsub_ru(v, b.L);
    float c = fmaxf(ceilf(__fdiv_ru(r, b.delta)), 1.0f);
    if (c <= 255.0f && __fmul_rd(c, b.delta) < r) c += 1.0f;
    if (!(c <= 255.0f)) {
        off = true;
        return 255u;
    }
    return (unsigned)c;
}

// The MIP-bound texel of cell slice sl at (x, y): the codes of planes sl - 1
// (low byte) and sl (high byte), clamped to the cube.
__device__ __forceinline__ unsigned short bound_texel(const float* __restrict__ bricks,
                                                      const VolumeGeom& g, const BoundScale& b,
                                                      int x, int y, int sl, bool& off)
{
    const int za = min(max(sl - 1, 0), g.nz - 1), zb = min(sl, g.nz - 1);
    const unsigned lo = bound_code(bricks[voxel_index(g, x, y, za)], b, off);
    const unsigned hi = bound_code(bricks[voxel_index(g, x, y, zb)], b, off);
    return (unsigned short)(lo | (hi << 8));
}

// A voxel without a code turns skipping off for good (until the scale is
// derived again): every sample becomes a candidate.
__device__ __forceinline__ void bound_disable(bool off, BoundScale* __restrict__ b)
{
    if (__syncthreads_or(off) && threadIdx.x == 0) b->le = INFINITY;
}

// MIP bounds: cell slices [s0, s1) (slice s holds planes s - 1 and s, s in
// [0, nz]) through a surface, stacked as the FP32 texture's slices.
__global__ void __launch_bounds__(256) fill_bound_kernel(const float* __restrict__ bricks,
                                                         VolumeGeom g, cudaSurfaceObject_t surf,
                                                         int s0, int s1, int shift, int pitch,
                                                         BoundScale* __restrict__ bs)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const BoundScale b = *bs;
    bool off = false;
    if (x < g.nx && y < g.ny) {
        for (int sl = s0 + blockIdx.z; sl < s1; sl += gridDim.z)
            write_slice_row(surf, bound_texel(bricks, g, b, x, y, sl, off), x, y, sl, g.ny,
                            shift, pitch);
    }
    bound_disable(off, bs);
}

// fill_bound_kernel's slices written linearly: slice s0 + j at dst + j nx ny,
// x fastest (for a copy into an unstacked bound texture).
__global__ void __launch_bounds__(256) fill_bound_linear_kernel(
    const float* __restrict__ bricks, VolumeGeom g, unsigned short* __restrict__ dst, int s0,
    int s1, BoundScale* __restrict__ bs)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const BoundScale b = *bs;
    bool off = false;
    if (x < g.nx && y < g.ny) {
        for (int sl = s0 + blockIdx.z; sl < s1; sl += gridDim.z)
            dst[((size_t)(sl - s0) * g.ny + y) * g.nx + x] =
                bound_texel(bricks, g, b, x, y, sl, off);
    }
    bound_disable(off, bs);
}

// Pair formats: slices [s0, s1); slice s holds the voxels of planes s - 1 and
// s (clamped to the cube) packed in one texel, low bits plane s - 1.  `flip`
// is XORed into the packed texel: int8 codes are stored as q + 128 (each
// byte's sign bit flipped), which the march turns back into q exactly
// (vr_ray.cuh, code_lo).
template <typename T, typename W>
__global__ void __launch_bounds__(256) fill_pair_kernel(const T* __restrict__ bricks, VolumeGeom g,
                                                        cudaSurfaceObject_t surf, int s0, int s1,
                                                        int shift, int pitch, W flip)
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
        const W packed = (W)(((W)(unsigned)(typename std::make_unsigned<T>::type)lo |
                              ((W)(unsigned)(typename std::make_unsigned<T>::type)hi
                               << (8 * sizeof(T)))) ^ flip);
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
    if (pair)   // {scale, scale, offset, offset} of planes sl - 1 and sl
        static_cast<float4*>(out)[sl] = make_float4(scale[z0], scale[z1], offset[z0], offset[z1]);
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

// The bound kernels' grid: 32 x 8 voxel rows per block, at most 32 blocks
// along the slices (each block then walks several slices), so that the
// range reduction takes a few thousand atomics rather than one per warp row.
static dim3 bound_grid(const Volume& v, int z0, int z1)
{
    return dim3((unsigned)((v.g.nx + 31) / 32), (unsigned)((v.g.ny + 7) / 8),
                (unsigned)std::max(1, std::min(z1 - z0, 32)));
}

cudaError_t bound_scale(const Volume& v, cudaStream_t s)
{
    bound_reset_kernel<<<1, 1, 0, s>>>(v.bound_scale);
    bound_range_kernel<<<bound_grid(v, 0, v.g.nz), 256, 0, s>>>((const float*)v.bricks, v.g,
                                                                v.bound_scale);
    bound_finish_kernel<<<1, 1, 0, s>>>(v.bound_scale);
    return cudaGetLastError();
}

cudaError_t fill_bounds(const Volume& v, cudaSurfaceObject_t surf, int z0, int z1,
                        cudaStream_t s)
{
    if (z1 <= z0) return cudaSuccess;
    const dim3 grid = bound_grid(v, z0, z1);
    fill_bound_kernel<<<grid, 256, 0, s>>>((const float*)v.bricks, v.g, surf, z0, z1,
                                           v.stack_shift, v.stack_pitch, v.bound_scale);
    return cudaGetLastError();
}

cudaError_t fill_bounds_linear(const Volume& v, unsigned short* dst, int z0, int z1,
                               cudaStream_t s)
{
    if (z1 <= z0) return cudaSuccess;
    const dim3 grid = bound_grid(v, z0, z1);
    fill_bound_linear_kernel<<<grid, 256, 0, s>>>((const float*)v.bricks, v.g, dst, z0, z1,
                                                  v.bound_scale);
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
            (const unsigned short*)v.bricks, v.g, surf, z0, z1, sh, pt, 0u);
        return cudaGetLastError();
    }
    if (v.tex_format == kI8Pair) {
        fill_pair_kernel<signed char, unsigned short><<<grid, 256, 0, s>>>(
            (const signed char*)v.bricks, v.g, surf, z0, z1, sh, pt, (unsigned short)0x8080u);
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
