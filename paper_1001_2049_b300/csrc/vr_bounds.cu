// vr_bounds.cu -- the empty-space bounds grid of a volume.
//
// The clip of the transfer function (samples below it are fully
// transparent, the reading of the paper's emphasis on low signal-to-noise
// data, abstract and §3.1 item 3) leaves most samples of a noise-dominated
// cube without effect, and so does every sample of a MIP ray that is not
// above the ray's running maximum.  The bounds grid lets the march pass over
// such samples without fetching them: one float per macrocell of 4^3 cells
// (voxels [4m, 4m + 4] per axis, the cells' corners), at least the largest
// value the kernels can compute for a sample in it.
//
// The kernels' value of a sample is three levels of lerp (fma(f, b - a, a),
// f in [0, 1]) over the decoded corners.  One level can exceed the larger of
// its two inputs by at most 3u max|corner| (u = 2^-24: the rounding of b - a
// and of the fma), so three levels by less than 10u max|corner|.  The bound
// stored is max + 2^-19 max|corner| (32u), rounded once by an fma, which
// stays above that.  Decoding is the kernels' own: float32 as stored,
// binary16 widened exactly, int8 as fma(code, scale[z], offset[z]).
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

// One thread per macrocell; 64 macrocells along x by 4 along y per block,
// one macrocell plane per grid z.
template <int DT>
__global__ void __launch_bounds__(256) bound_kernel(const void* __restrict__ bricks,
                                                    const float* __restrict__ scale,
                                                    const float* __restrict__ offset,
                                                    VolumeGeom g, float* __restrict__ out,
                                                    int bnx, int bny, int mz0)
{
    const int mx = blockIdx.x * 64 + (threadIdx.x & 63);
    const int my = blockIdx.y * 4 + (threadIdx.x >> 6);
    const int mz = mz0 + (int)blockIdx.z;
    if (mx >= bnx || my >= bny) return;
    const int x0 = mx << kMacroShift, x1 = min(x0 + kMacro, g.nx - 1);
    const int y0 = my << kMacroShift, y1 = min(y0 + kMacro, g.ny - 1);
    const int z0 = mz << kMacroShift, z1 = min(z0 + kMacro, g.nz - 1);
    float hi = -INFINITY, mag = 0.0f;
    for (int z = z0; z <= z1; ++z) {
        float s = 1.0f, o = 0.0f;
        if (DT == VR_I8) {
            s = __ldg(scale + z);
            o = __ldg(offset + z);
        }
        for (int y = y0; y <= y1; ++y) {
            const size_t row = ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx;
            const size_t in = (size_t)((z & 31) << 10) + ((y & 31) << 5);
            for (int x = x0; x <= x1; ++x) {
                float v = voxel<DT>(bricks, (row + (x >> kBrickShift)) * kBrickVoxels + in +
                                                (x & 31));
                if (DT == VR_I8) v = fmaf(v, s, o);
                hi = fmaxf(hi, v);
                mag = fmaxf(mag, fabsf(v));
            }
        }
    }
    out[((size_t)mz * bny + my) * bnx + mx] = fmaf(mag, 0x1p-19f, hi);
}

}  // namespace

cudaError_t launch_bounds(const Volume& v, int mz0, int mz1, cudaStream_t s)
{
    for (; mz1 - mz0 > 65535; mz0 += 65535) {           // grid z limit
        const cudaError_t e = launch_bounds(v, mz0, mz0 + 65535, s);
        if (e != cudaSuccess) return e;
    }
    if (mz1 <= mz0) return cudaSuccess;
    const dim3 grid((unsigned)((v.bnx + 63) / 64), (unsigned)((v.bny + 3) / 4),
                    (unsigned)(mz1 - mz0));
    switch (v.dtype) {
    case VR_F32:
        bound_kernel<VR_F32><<<grid, 256, 0, s>>>(v.bricks, v.scale, v.offset, v.g, v.bound,
                                                  v.bnx, v.bny, mz0);
        break;
    case VR_F16:
        bound_kernel<VR_F16><<<grid, 256, 0, s>>>(v.bricks, v.scale, v.offset, v.g, v.bound,
                                                  v.bnx, v.bny, mz0);
        break;
    default:
        bound_kernel<VR_I8><<<grid, 256, 0, s>>>(v.bricks, v.scale, v.offset, v.g, v.bound,
                                                 v.bnx, v.bny, mz0);
        break;
    }
    return cudaGetLastError();
}

}  // namespace vr
