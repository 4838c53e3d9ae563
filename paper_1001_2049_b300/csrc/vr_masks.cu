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

// One block of 64 threads per macrocell, thread t the cell
// (t & 3, (t >> 2) & 3, t >> 4) of it.
template <int DT>
__global__ void __launch_bounds__(64) mask_kernel(const void* __restrict__ bricks,
                                                  const float* __restrict__ scale,
                                                  const float* __restrict__ offset,
                                                  VolumeGeom g, unsigned* __restrict__ out,
                                                  int mnx, int mny, float clip)
{
    const unsigned m = blockIdx.x;
    const int mx = (int)(m % mnx), my = (int)((m / mnx) % mny), mz = (int)(m / ((unsigned)mnx * mny));
    const int t = threadIdx.x;
    const int gx = (mx << kMacroShift) + (t & 3);           // gather coordinates: cell + 1
    const int gy = (my << kMacroShift) + ((t >> 2) & 3);
    const int gz = (mz << kMacroShift) + (t >> 4);
    bool need = false;
    if (gx <= g.nx && gy <= g.ny && gz <= g.nz) {
        const int cx = min(max(gx - 1, 0), g.nx - 2);
        const int cy = min(max(gy - 1, 0), g.ny - 2);
        const int cz = min(max(gz - 1, 0), g.nz - 2);
        float hi = -INFINITY, mag = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int x = cx + (c & 1), y = cy + ((c >> 1) & 1), z = cz + (c >> 2);
            const size_t brick =
                ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx + (x >> kBrickShift);
            float v = voxel<DT>(bricks, brick * kBrickVoxels + ((z & 31) << 10) + ((y & 31) << 5) +
                                            (x & 31));
            if (DT == VR_I8) v = fmaf(v, __ldg(scale + z), __ldg(offset + z));
            hi = fmaxf(hi, v);
            mag = fmaxf(mag, fabsf(v));
        }
        need = !(fmaf(mag, 0x1p-19f, hi) < clip);
    }
    const unsigned word = __ballot_sync(0xffffffffu, need);
    if ((t & 31) == 0) out[2 * (size_t)m + (t >> 5)] = word;
}

}  // namespace

cudaError_t launch_masks(const Volume& v, float clip, cudaStream_t s)
{
    const unsigned nm = (unsigned)v.mnx * v.mny * v.mnz;
    unsigned* out = reinterpret_cast<unsigned*>(v.mask);
    switch (v.dtype) {
    case VR_F32:
        mask_kernel<VR_F32><<<nm, 64, 0, s>>>(v.bricks, v.scale, v.offset, v.g, out, v.mnx, v.mny,
                                              clip);
        break;
    case VR_F16:
        mask_kernel<VR_F16><<<nm, 64, 0, s>>>(v.bricks, v.scale, v.offset, v.g, out, v.mnx, v.mny,
                                              clip);
        break;
    default:
        mask_kernel<VR_I8><<<nm, 64, 0, s>>>(v.bricks, v.scale, v.offset, v.g, out, v.mnx, v.mny,
                                             clip);
        break;
    }
    return cudaGetLastError();
}

}  // namespace vr
