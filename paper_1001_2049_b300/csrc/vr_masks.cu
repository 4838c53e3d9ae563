// vr_masks.cu -- the empty-space masks of a volume.
//
// The clip of the transfer function (samples below it are fully
// transparent, the reading of the paper's emphasis on low signal-to-noise
// data, abstract and §3.1 item 3) leaves most samples of a noise-dominated
// cube without effect.  The masks let the composite march tell such samples
// from the rest without fetching them: per macrocell of 4 x 4 x 4 cells, a
// 64-bit mask of the cells that can hold a visible sample for the current
// clip level, built on the render stream whenever the clip changes.
//
// A cell's bit is clear only when every value the kernels can interpolate in
// it is below the clip.  That value is three levels of lerp (fma(f, b - a,
// a), f in [0, 1]) over the cell's eight decoded corners; one level can
// exceed the larger of its two inputs by at most 3u max|corner| (u = 2^-24:
// the rounding of b - a and of the fma), three levels by less than
// 10u max|corner|.  The bit is clear when max + 2^-19 max|corner| (32u,
// rounded once by an fma) is below the clip.  Decoding is the kernels' own:
// float32 as stored, binary16 widened exactly, int8 as fma(code, scale[z],
// offset[z]).
//
// Cells are indexed by the kernels' gather coordinates: on every axis from
// -1 to n - 1 (stored at +1; the outermost cells hold positions a rounding
// error outside the box, which read the edge voxels, so they take the bit of
// the edge cell).
#include <cuda_fp16.h>

#include "vr_internal.h"

namespace vr {
namespace {

template <int DT>
__device__ __forceinline__ float voxel(const void* __restrict__ b, size_t i)
{
    if (DT == VR_F32) return __ldg(static_cast<const float*>(b) + i);
    if (DT == VR_F16) return __half2float(__ldg(static_cast<const __half*>(b) + i));
    return (float)__ldg(static_cast<const signed char*>(b) + i);
}

// One block of 16 warps per column of 8 x 1 macrocells (walked along z):
// for each macrocell row, warp w takes cell
// row (y, z) = (w & 3, w >> 2) of the macrocells, lane l the cell at gather
// coordinate x = 32 bx + l.  The block's corner voxels (33 x 5 x 5, indices
// clamped to the cube) are staged once in shared memory, decoded.
// A warp's ballot holds 4 x-bits of each of the 8 macrocells for its (y, z);
// eight threads assemble the masks from the 16 ballots.
constexpr int kMaskWarps = 16;
constexpr int kTileX = 33, kTileYZ = 5;

template <int DT>
__global__ void __launch_bounds__(32 * kMaskWarps) mask_kernel(
    const void* __restrict__ bricks, const float* __restrict__ scale,
    const float* __restrict__ offset, VolumeGeom g, unsigned long long* __restrict__ out,
    int mnx, int mny, int mnz, float clip)
{
    __shared__ float s_v[kTileYZ][kTileYZ][kTileX];
    __shared__ unsigned s_ballot[kMaskWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // tile origin: the block's first cell, clamped like every cell (the
    // clamped cells of the block then lie in [origin, origin + 31] along x
    // and [origin, origin + 3] along y and z, clamping being 1-Lipschitz)
    const int x0 = min(max((int)blockIdx.x * 32 - 1, 0), g.nx - 2);
    const int y0 = min(max((int)blockIdx.y * 4 - 1, 0), g.ny - 2);
    const int gx = blockIdx.x * 32 + lane;                      // gather coordinates: cell + 1
    const int gy = blockIdx.y * 4 + (w & 3);
    // one row of macrocells along z after the other (the block walks its
    // column, so the launch has few blocks)
    for (int bz = 0; bz < mnz; ++bz) {
        const int z0 = min(max(bz * 4 - 1, 0), g.nz - 2);
        __syncthreads();                 // the previous row's tile and ballots are used up
        for (int i = threadIdx.x; i < kTileX * kTileYZ * kTileYZ; i += 32 * kMaskWarps) {
            const int tx = i % kTileX, ty = (i / kTileX) % kTileYZ, tz = i / (kTileX * kTileYZ);
            const int x = min(x0 + tx, g.nx - 1);
            const int y = min(y0 + ty, g.ny - 1);
            const int z = min(z0 + tz, g.nz - 1);
            const size_t brick = ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx +
                                 (x >> kBrickShift);
            float v = voxel<DT>(bricks, brick * kBrickVoxels + ((z & 31) << 10) + ((y & 31) << 5) +
                                            (x & 31));
            if (DT == VR_I8) v = fmaf(v, __ldg(scale + z), __ldg(offset + z));
            s_v[tz][ty][tx] = v;
        }
        __syncthreads();
        const int gz = bz * 4 + (w >> 2);
        bool need = false;
        if (gx <= g.nx && gy <= g.ny && gz <= g.nz) {
            // the cell's corners, as tile indices (cells clamped to the cube)
            const int cx = min(max(gx - 1, 0), g.nx - 2) - x0;
            const int cy = min(max(gy - 1, 0), g.ny - 2) - y0;
            const int cz = min(max(gz - 1, 0), g.nz - 2) - z0;
            float hi = -INFINITY, mag = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float v = s_v[cz + (c >> 2)][cy + ((c >> 1) & 1)][cx + (c & 1)];
                hi = fmaxf(hi, v);
                mag = fmaxf(mag, fabsf(v));
            }
            need = !(fmaf(mag, 0x1p-19f, hi) < clip);
        }
        const unsigned b = __ballot_sync(0xffffffffu, need);
        if (lane == 0) s_ballot[w] = b;
        __syncthreads();
        if (threadIdx.x < 8) {
            const int mx = blockIdx.x * 8 + threadIdx.x;
            if (mx < mnx) {
                unsigned long long m = 0;
#pragma unroll
                for (int i = 0; i < kMaskWarps; ++i) {
                    const unsigned long long nib = (s_ballot[i] >> (4 * threadIdx.x)) & 0xfu;
                    m |= nib << (4 * (i & 3) + 16 * (i >> 2));      // bit x | y << 2 | z << 4
                }
                out[((size_t)bz * mny + blockIdx.y) * mnx + mx] = m;
            }
        }
    }
}

}  // namespace

cudaError_t launch_masks(const Volume& v, float clip, cudaStream_t s)
{
    const dim3 grid((unsigned)((v.mnx + 7) / 8), (unsigned)v.mny);
    switch (v.dtype) {
    case VR_F32:
        mask_kernel<VR_F32><<<grid, 32 * kMaskWarps, 0, s>>>(v.bricks, v.scale, v.offset, v.g,
                                                             v.mask, v.mnx, v.mny, v.mnz, clip);
        break;
    case VR_F16:
        mask_kernel<VR_F16><<<grid, 32 * kMaskWarps, 0, s>>>(v.bricks, v.scale, v.offset, v.g,
                                                             v.mask, v.mnx, v.mny, v.mnz, clip);
        break;
    default:
        mask_kernel<VR_I8><<<grid, 32 * kMaskWarps, 0, s>>>(v.bricks, v.scale, v.offset, v.g,
                                                            v.mask, v.mnx, v.mny, v.mnz, clip);
        break;
    }
    return cudaGetLastError();
}

}  // namespace vr
