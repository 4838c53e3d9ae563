// vr_pack.cu -- packing a linear float32 spectral cube into 32^3 bricks, with
// conversion to the storage type.
//
// Paper §3.1 process item 1 partitions the cube into sub-cubes; here the
// partition is the on-device brick layout: bricks in brick-major order (bx
// fastest, then by, then bz), voxels inside a brick x fastest, then y, then
// z.  Dims that are not multiples of 32 are zero-padded; the padding is never
// sampled because the render box ends at the last voxel centre.
//
// Storage types: float32 as given; float16 round-to-nearest-even; int8 with a
// scale and offset per frequency plane z (lo = min, hi = max over the plane,
// scale = (hi - lo)/254, offset = (hi + lo)/2, code = clamp(rint((v -
// offset)/scale), -127, 127), every step in float32 with IEEE rounding so
// the codes are reproducible; a constant plane gets scale 1 and code 0).
//
// Both kernels are HBM-bound one-time copies (not part of the render path).
#include <cuda_fp16.h>

#include "vr_internal.h"

namespace vr {
namespace {

template <int DT>
struct Enc;

template <>
struct Enc<VR_F32> {
    using T = float;
    __device__ static T code(float v, float, float) { return v; }
    __device__ static T zero() { return 0.0f; }
};

template <>
struct Enc<VR_F16> {
    using T = __half;
    __device__ static T code(float v, float, float) { return __float2half_rn(v); }
    __device__ static T zero() { return __float2half_rn(0.0f); }
};

template <>
struct Enc<VR_I8> {
    using T = int8_t;
    __device__ static T code(float v, float scale, float offset) {
        float r = __fdiv_rn(__fsub_rn(v, offset), scale);
        float q = fminf(fmaxf(rintf(r), -127.0f), 127.0f);
        return (int8_t)(int)q;
    }
    __device__ static T zero() { return 0; }
};

// Per-plane min and max -> scale/offset for planes [z0, z0 + nplanes).
// One block per plane (grid-stride over planes).
__global__ void __launch_bounds__(512) plane_scale_kernel(
    const float* __restrict__ src, float* __restrict__ scale, float* __restrict__ offset,
    VolumeGeom g, int z0, int nplanes)
{
    __shared__ float s_lo[16], s_hi[16];
    const size_t plane = (size_t)g.nx * g.ny;
    for (int zr = blockIdx.x; zr < nplanes; zr += gridDim.x) {
        const float* p = src + (size_t)zr * plane;
        float lo = INFINITY, hi = -INFINITY;
        for (size_t i = threadIdx.x; i < plane; i += blockDim.x) {
            float v = p[i];
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) {
            s_lo[warp] = lo;
            s_hi[warp] = hi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                lo = fminf(lo, s_lo[w]);
                hi = fmaxf(hi, s_hi[w]);
            }
            float sc = (hi == lo) ? 1.0f : __fdiv_rn(__fsub_rn(hi, lo), 254.0f);
            float of = __fmul_rn(__fadd_rn(hi, lo), 0.5f);
            scale[z0 + zr] = sc;
            offset[z0 + zr] = of;
        }
        __syncthreads();
    }
}

// Writes the brick slabs of planes [z0, z_end): voxels with z < z_src_end
// come from src (which starts at plane z0), the rest (x/y/z padding) are 0.
// grid.x = one 32x32 brick slab of a plane, grid.y strides over planes.
template <int DT>
__global__ void __launch_bounds__(256) pack_kernel(
    const float* __restrict__ src, typename Enc<DT>::T* __restrict__ dst,
    const float* __restrict__ scale, const float* __restrict__ offset, VolumeGeom g,
    int z0, int z_src_end, int z_end)
{
    using T = typename Enc<DT>::T;
    const int bx = blockIdx.x % g.nbx;
    const int by = blockIdx.x / g.nbx;
    for (int z = z0 + blockIdx.y; z < z_end; z += gridDim.y) {
        const size_t brick = ((size_t)(z >> kBrickShift) * g.nby + by) * g.nbx + bx;
        T* d = dst + brick * kBrickVoxels + (size_t)(z & 31) * (kBrick * kBrick);
        float sc = 1.0f, of = 0.0f;
        if (DT == VR_I8 && z < z_src_end) {
            sc = scale[z];
            of = offset[z];
        }
        for (int e = threadIdx.x; e < kBrick * kBrick; e += blockDim.x) {
            const int x = bx * kBrick + (e & 31);
            const int y = by * kBrick + (e >> 5);
            T out = Enc<DT>::zero();
            if (x < g.nx && y < g.ny && z < z_src_end) {
                const float v = src[((size_t)(z - z0) * g.ny + y) * g.nx + x];
                out = Enc<DT>::code(v, sc, of);
            }
            d[e] = out;
        }
    }
}

}  // namespace

cudaError_t launch_pack(const Volume& v, int64_t z0, int64_t nplanes, const float* src,
                        cudaStream_t s)
{
    const VolumeGeom& g = v.g;
    const int zs = (int)z0;
    const int z_src_end = (int)(z0 + nplanes);
    // the chunk that ends the cube also zero-fills the padding planes
    const int z_end = (z_src_end == g.nz) ? g.nbz * kBrick : z_src_end;
    if (v.dtype == VR_I8) {
        int grid = (int)(nplanes < 65535 ? nplanes : 65535);
        plane_scale_kernel<<<grid, 512, 0, s>>>(src, v.scale, v.offset, g, zs, (int)nplanes);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)(g.nbx * g.nby), (unsigned)((z_end - zs) < 65535 ? (z_end - zs) : 65535));
    switch (v.dtype) {
    case VR_F32:
        pack_kernel<VR_F32><<<grid, 256, 0, s>>>(src, (float*)v.bricks, v.scale, v.offset, g,
                                                 zs, z_src_end, z_end);
        break;
    case VR_F16:
        pack_kernel<VR_F16><<<grid, 256, 0, s>>>(src, (__half*)v.bricks, v.scale, v.offset, g,
                                                 zs, z_src_end, z_end);
        break;
    default:
        pack_kernel<VR_I8><<<grid, 256, 0, s>>>(src, (int8_t*)v.bricks, v.scale, v.offset, g,
                                                zs, z_src_end, z_end);
        break;
    }
    return cudaGetLastError();
}

}  // namespace vr
