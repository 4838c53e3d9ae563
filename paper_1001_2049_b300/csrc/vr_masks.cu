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
// offset[z]).  int8 textures interpolate the codes of each plane and
// decode that (interp_t): the codes' two lerp levels err by at most 512u
// code units (|code| <= 127), i.e. 512u |scale| once decoded, which a further
// 2^-14 max |scale| of the cell's two planes covers.
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

// One block of 4 warps per column of 8 x 1 macrocells (32 x 4 cells across),
// walked along z in chunks of kRows macrocell rows.  The chunk's corner voxels
// (33 x 5 x (4 kRows + 1), indices clamped to the cube) are staged in shared
// memory, decoded.  FP32 cubes stage with asynchronous 4-byte copies into two
// buffers, the next chunk's copies in flight while the current chunk is
// tested; FP16 and int8 cubes (elements too small for those copies) issue all
// of a chunk's loads before storing any (about 22 in flight per thread), then
// decode and store them.  Thread (lane, warp) owns the cell column at gather
// coordinates x = 32 bx + lane, y = 4 by + warp and walks it along z: the
// largest value and the largest |value| of a plane's 2 x 2 corners are
// computed once and serve the two cells that plane bounds, so a step reads
// the four corners of one new plane.  A warp's ballot holds 4 x-bits of each
// of the 8 macrocells for its (y, z); after the chunk, 8 x kRows threads
// assemble the masks from the ballots.
constexpr int kMaskWarps = 4;
constexpr int kRows = 4;
constexpr int kTileX = 33, kTileY = 5, kTileZ = 4 * kRows + 1;
constexpr int kTileElems = kTileX * kTileY * kTileZ;
constexpr int kMaskThreads = 32 * kMaskWarps;
constexpr int kPerThread = (kTileElems + kMaskThreads - 1) / kMaskThreads;

// Brick-layout index of tile element i of the chunk whose tile origin is
// (x0, y0, z0); element i = (tz * 5 + ty) * 33 + tx, indices clamped.
__device__ __forceinline__ size_t tile_voxel(const VolumeGeom& g, int x0, int y0, int z0, int i,
                                             int* zout)
{
    const int row = i / kTileX, tx = i - row * kTileX;
    const int tz = row / kTileY, ty = row - tz * kTileY;
    const int x = min(x0 + tx, g.nx - 1);
    const int y = min(y0 + ty, g.ny - 1);
    const int z = min(z0 + tz, g.nz - 1);
    *zout = z;
    const size_t brick = ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) * g.nbx +
                         (x >> kBrickShift);
    return brick * kBrickVoxels + ((z & 31) << 10) + ((y & 31) << 5) + (x & 31);
}

__device__ __forceinline__ void copy_async4(float* dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

template <int DT>
__global__ void __launch_bounds__(kMaskThreads) mask_kernel(
    const void* __restrict__ bricks, const float* __restrict__ scale,
    const float* __restrict__ offset, VolumeGeom g, unsigned long long* __restrict__ out,
    int mnx, int mny, int mnz, float clip)
{
    constexpr int kBufs = DT == VR_F32 ? 2 : 1;
    __shared__ float s_v[kBufs][kTileZ][kTileY][kTileX];
    __shared__ unsigned s_ballot[4 * kRows][kMaskWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // tile origin: the block's first cell (the chunk's along z), clamped
    // like every cell (the clamped cells then lie in [origin, origin + 31]
    // along x, [origin, origin + 3] along y and [origin, origin + 4 kRows -
    // 1] along z, clamping being 1-Lipschitz)
    const int x0 = min(max((int)blockIdx.x * 32 - 1, 0), g.nx - 2);
    const int y0 = min(max((int)blockIdx.y * 4 - 1, 0), g.ny - 2);
    const int gx = blockIdx.x * 32 + lane;                      // gather coordinates: cell + 1
    const int gy = blockIdx.y * 4 + w;
    const bool in_xy = gx <= g.nx && gy <= g.ny;
    // the cell's corner columns and rows, as tile indices (cells clamped)
    const int cx = min(max(gx - 1, 0), g.nx - 2) - x0;
    const int cy = min(max(gy - 1, 0), g.ny - 2) - y0;
    auto chunk_z0 = [&](int bz0) { return min(max(bz0 * 4 - 1, 0), g.nz - 2); };
    // FP32: copies of chunk bz0 into buffer b (one commit group), a tile row
    // (fixed y, z) per warp step: lane l copies column l, lane 0 also column
    // 32; a column's offset inside a brick row is the same for every row
    const int col_a = min(x0 + lane, g.nx - 1), col_b = min(x0 + 32, g.nx - 1);
    const size_t off_a = (size_t)(col_a >> kBrickShift) * kBrickVoxels + (col_a & 31);
    const size_t off_b = (size_t)(col_b >> kBrickShift) * kBrickVoxels + (col_b & 31);
    auto stage_async = [&](int b, int bz0) {
        const int z0 = chunk_z0(bz0);
        float* dst = &s_v[b][0][0][0];
        const float* src = static_cast<const float*>(bricks);
        for (int r = w; r < kTileZ * kTileY; r += kMaskWarps) {
            const int tz = r / kTileY, ty = r - tz * kTileY;
            const int y = min(y0 + ty, g.ny - 1);
            const int z = min(z0 + tz, g.nz - 1);
            const size_t row = ((size_t)(z >> kBrickShift) * g.nby + (y >> kBrickShift)) *
                                   g.nbx * kBrickVoxels +
                               ((z & 31) << 10) + ((y & 31) << 5);
            copy_async4(dst + r * kTileX + lane, src + row + off_a);
            if (lane == 0) copy_async4(dst + r * kTileX + 32, src + row + off_b);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if constexpr (DT == VR_F32) stage_async(0, 0);
    for (int bz0 = 0, j = 0; bz0 < mnz; bz0 += kRows, ++j) {
        const int z0 = chunk_z0(bz0);
        const int b = kBufs == 2 ? (j & 1) : 0;
        if constexpr (DT == VR_F32) {
            // the next chunk's copies go to the other buffer (free: its last
            // use ended before the barrier closing the previous chunk); then
            // wait for this chunk's
            if (bz0 + kRows < mnz) {
                stage_async(b ^ 1, bz0 + kRows);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();
        } else {
            // all loads first, then decode and store
            float vals[kPerThread];
            int zs[kPerThread];
#pragma unroll
            for (int k = 0; k < kPerThread; ++k) {
                const int i = threadIdx.x + k * kMaskThreads;
                if (i < kTileElems) vals[k] = voxel<DT>(bricks, tile_voxel(g, x0, y0, z0, i, &zs[k]));
            }
            __syncthreads();             // the previous chunk's tile and ballots are used up
            float* s_flat = &s_v[0][0][0][0];
#pragma unroll
            for (int k = 0; k < kPerThread; ++k) {
                const int i = threadIdx.x + k * kMaskThreads;
                if (i < kTileElems) {
                    float v = vals[k];
                    if (DT == VR_I8) v = fmaf(v, __ldg(scale + zs[k]), __ldg(offset + zs[k]));
                    s_flat[i] = v;
                }
            }
            __syncthreads();
        }
        // walk the chunk's cells along z; a plane's corner bounds serve the
        // cell below and the cell above it
        int have = -1;                   // tile plane whose bounds are in hi1 / mag1
        float hi0 = 0.0f, mag0 = 0.0f, sc0 = 0.0f, hi1 = 0.0f, mag1 = 0.0f, sc1 = 0.0f;
        auto plane_bounds = [&](int pz, float& hi, float& mag, float& sc) {
            const float a = s_v[b][pz][cy][cx], bb = s_v[b][pz][cy][cx + 1];
            const float c = s_v[b][pz][cy + 1][cx], d = s_v[b][pz][cy + 1][cx + 1];
            // (fmaxf ignores NaN; the -inf and 0 keep a plane of NaN corners
            // from giving a NaN bound)
            hi = fmaxf(fmaxf(fmaxf(a, bb), fmaxf(c, d)), -INFINITY);
            mag = fmaxf(fmaxf(fmaxf(fabsf(a), fabsf(bb)), fmaxf(fabsf(c), fabsf(d))), 0.0f);
            sc = DT == VR_I8 ? 0x1p-14f * fabsf(__ldg(scale + min(z0 + pz, g.nz - 1))) : 0.0f;
        };
        for (int c = 0; c < 4 * kRows; ++c) {
            const int gz = bz0 * 4 + c;
            // block-uniform: the cell's lower plane in the tile
            const int cz = min(max(gz - 1, 0), g.nz - 2) - z0;
            if (cz == have) {            // the next plane up: its lower plane is held
                hi0 = hi1;
                mag0 = mag1;
                sc0 = sc1;
                plane_bounds(cz + 1, hi1, mag1, sc1);
                have = cz + 1;
            } else if (cz + 1 != have) { // first cell of the chunk
                plane_bounds(cz, hi0, mag0, sc0);
                plane_bounds(cz + 1, hi1, mag1, sc1);
                have = cz + 1;
            }                            // else: the same cell again (clamped at an edge)
            const bool need = in_xy && gz <= g.nz &&
                              !(fmaf(fmaxf(mag0, mag1), 0x1p-19f,
                                     fmaxf(hi0, hi1) + fmaxf(sc0, sc1)) < clip);
            const unsigned bal = __ballot_sync(0xffffffffu, need);
            if (lane == 0) s_ballot[c][w] = bal;
        }
        __syncthreads();
        // masks of the chunk's 8 x kRows macrocells
        if (threadIdx.x < 8 * kRows) {
            const int mx = blockIdx.x * 8 + (threadIdx.x & 7);
            const int bz = bz0 + (threadIdx.x >> 3);
            if (mx < mnx && bz < mnz) {
                const int c0 = (threadIdx.x >> 3) * 4, sh = 4 * (threadIdx.x & 7);
                unsigned long long m = 0;
#pragma unroll
                for (int i = 0; i < 16; ++i) {   // cell row y = i & 3, z = i >> 2
                    const unsigned long long nib = (s_ballot[c0 + (i >> 2)][i & 3] >> sh) & 0xfu;
                    m |= nib << (4 * i);                        // bit x | y << 2 | z << 4
                }
                out[((size_t)bz * mny + blockIdx.y) * mnx + mx] = m;
            }
        }
        __syncthreads();                 // this chunk's buffer and ballots are used up
    }
}

}  // namespace

cudaError_t launch_masks(const Volume& v, float clip, cudaStream_t s)
{
    const dim3 grid((unsigned)((v.mnx + 7) / 8), (unsigned)v.mny);   // 32 x 4 cells each
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
